"""The allocation-free V-cycle entry point (sg_vcycle_apply_static).

Callers that must not allocate device memory while they run (inside a stream
capture, an allocator hook, or a fixed memory budget) use this entry point; it
keeps its buffers in a fixed array inside the library. The test calls it
through the C ABI twice in a row and checks each result against the regular
sg_vcycle_apply on the same input. It sits in a file of its own, collected
last, and passes both alone in a fresh process and after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

import sg_inputs as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [("f32", 2e-6), ("f64", 1e-13)])
def test_static_vcycle_matches_regular_on_two_calls(prec, tol):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1205_1864_gb300 as L
    from paper_1205_1864_gb300 import _lib

    dt = torch.float32 if prec == "f32" else torch.float64
    code = L.SG_F32 if prec == "f32" else L.SG_F64
    prob = S.make_problem(64, 2, 0.3, 0.5)           # 63 x 63 interior grid: grid kernels and the coarse block
    h = L.SGProblem.from_inputs(prob, 2)
    opts = L.prec_opts(nu=2, omega=0.8)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (w, seed) in enumerate([(17, 1), (33, 2)]):
        B = torch.tensor(S.random_block(prob.n, w, seed=seed), dtype=dt, device="cuda")
        ref = L.sg_vcycle_apply(h, B, opts)
        X = torch.full_like(B, float("nan"))
        st = _lib.LIB.sg_vcycle_apply_static(h.h, C.c_void_p(B.data_ptr()), C.c_void_p(X.data_ptr()), w, code,
                                             C.byref(opts), stream)
        assert st == 0, _lib.LIB.sg_last_error().decode()
        torch.cuda.synchronize()
        x, r = X.double().cpu().numpy(), ref.double().cpu().numpy()
        scale = np.abs(r).max(axis=0, keepdims=True)
        assert np.all(np.abs(x - r) <= tol * scale), (call, np.abs(x - r).max())


def test_static_vcycle_rejects_oversized_batch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1205_1864_gb300 as L
    from paper_1205_1864_gb300 import _lib

    prob = S.make_problem(256, 1, 0.3, 0.5)          # 65025 nodes: 1024 FP64 columns need far more than 32 MiB
    h = L.SGProblem.from_inputs(prob, 1)
    B = torch.zeros((prob.n, 1024), dtype=torch.float64, device="cuda")
    X = torch.empty_like(B)
    st = _lib.LIB.sg_vcycle_apply_static(h.h, C.c_void_p(B.data_ptr()), C.c_void_p(X.data_ptr()), 1024, L.SG_F64,
                                         C.byref(L.prec_opts()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 1
    assert "32" in _lib.LIB.sg_last_error().decode() or "scratch" in _lib.LIB.sg_last_error().decode()


def _scratch_bytes(grid_nodes, wp, es):
    """The scratch of one call as the header states it: wp ints and three
    blocks of n_g x wp elements per multigrid grid, each rounded up to 256 B."""
    a = lambda b: (b + 255) // 256 * 256
    return a(wp * 4) + sum(3 * a(n * wp * es) for n in grid_nodes)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_static_vcycle_widest_batch_that_fits(prec):
    """The widest batch the documented size admits on a 63 x 63 grid runs and
    matches sg_vcycle_apply (every carved view of the array in use, up to its
    end), and one column more is rejected."""
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1205_1864_gb300 as L
    from paper_1205_1864_gb300 import _lib

    dt = torch.float32 if prec == "f32" else torch.float64
    code = L.SG_F32 if prec == "f32" else L.SG_F64
    es, vw = (4, 4) if prec == "f32" else (8, 2)
    ne = 64
    grids, m = [], ne
    while m >= 2:
        grids.append((m - 1) ** 2)
        m //= 2
    cap = 32 << 20
    w = max(w for w in range(vw, 1025, vw) if _scratch_bytes(grids, w, es) <= cap)
    assert w < 1024 and _scratch_bytes(grids, w + vw, es) > cap
    prob = S.make_problem(ne, 2, 0.3, 0.5)
    h = L.SGProblem.from_inputs(prob, 2)
    opts = L.prec_opts(nu=2, omega=0.8)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    B = torch.tensor(S.random_block(prob.n, w + 1, seed=9), dtype=dt, device="cuda")
    ref = L.sg_vcycle_apply(h, B[:, :w].contiguous(), opts)
    Bw = B[:, :w].contiguous()
    X = torch.full_like(Bw, float("nan"))
    st = _lib.LIB.sg_vcycle_apply_static(h.h, C.c_void_p(Bw.data_ptr()), C.c_void_p(X.data_ptr()), w, code,
                                         C.byref(opts), stream)
    assert st == 0, _lib.LIB.sg_last_error().decode()
    torch.cuda.synchronize()
    x, r = X.double().cpu().numpy(), ref.double().cpu().numpy()
    tol = 2e-6 if prec == "f32" else 1e-13
    assert np.all(np.abs(x - r) <= tol * np.abs(r).max(axis=0, keepdims=True))
    X1 = torch.empty_like(B)
    st = _lib.LIB.sg_vcycle_apply_static(h.h, C.c_void_p(B.data_ptr()), C.c_void_p(X1.data_ptr()), w + 1, code,
                                         C.byref(opts), stream)
    assert st == 1
