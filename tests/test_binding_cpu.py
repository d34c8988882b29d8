"""The Python binding's argument checks, on the CPU: every call that hands a
block to the library as a bare pointer refuses a block whose shape or element
type differs from what the call reads or writes (the library would run past a
smaller tensor), and passes the shapes the tests and the benchmark use. The
library and the device are replaced by stand-ins that record the calls, so no
kernel runs."""
import importlib.util
import os
import types

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
F64, F32 = torch.float64, torch.float32


class FakeBlock:
    """Stands for a contiguous tensor: shape, dtype and device only."""

    def __init__(self, shape, dtype=F64, cuda=True):
        shape = (shape,) if isinstance(shape, int) else tuple(shape)
        self.shape, self.dtype, self.is_cuda, self.device = shape, dtype, cuda, "cuda" if cuda else "cpu"

    def is_contiguous(self):
        return True

    def data_ptr(self):
        return 0x1000


class FakeLib:
    """Every entry point returns SG_OK and records its name."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        if name == "sg_last_error":
            return lambda: b""

        def call(*args):
            self.calls.append(name)
            return 0
        return call


@pytest.fixture()
def L(monkeypatch):
    spec = importlib.util.spec_from_file_location(
        "sghsc_build", os.path.join(ROOT, "paper_1205_1864_gb300", "build.py"))
    B = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(B)
    B.build()
    import paper_1205_1864_gb300 as L
    fake_torch = types.SimpleNamespace(
        float64=F64, float32=F32,
        empty=lambda shape, dtype=F64, device=None: FakeBlock(shape, dtype),
        empty_like=lambda t: FakeBlock(t.shape, t.dtype, t.is_cuda),
        cuda=types.SimpleNamespace(current_stream=lambda: types.SimpleNamespace(cuda_stream=0)))
    monkeypatch.setattr(L, "torch", fake_torch)
    monkeypatch.setattr(L._lib, "LIB", FakeLib())
    return L


def _handle(L, M=3, p=3, n=49, q=-1):
    """A handle as the binding sees it (sizes and level offsets), no library object."""
    import math
    h = object.__new__(L.SGProblem)
    h.h = None
    h.n, h.M, h.p, h.q = n, M, p, q
    h.P = math.comb(M + p, M)
    h.nterm = M + 1 if q < 0 else math.comb(M + q, M)
    h.off = [0] + [math.comb(M + d, M) for d in range(p + 1)]
    return h


def test_products_take_the_documented_shapes(L):
    h = _handle(L)
    n, P = h.n, h.P
    for dt in (F64, F32):
        L.sg_apply(h, FakeBlock((n, P), dt))
        L.sg_apply(h, FakeBlock((n, P), dt), FakeBlock((n, P), dt))
    L.sg_apply(h, FakeBlock((n, P), F32), FakeBlock((n, P), F64), df64=True)
    L.sg_apply(h, FakeBlock((n, P), F32), df64=True)
    for bad in [((n, P - 1), F64, None), ((n + 1, P), F64, None), ((n, P), F64, ((n, P), F32)),
                ((n, P), F64, ((n, P + 1), F64))]:
        with pytest.raises(ValueError):
            L.sg_apply(h, FakeBlock(bad[0], bad[1]), None if bad[2] is None else FakeBlock(*bad[2]))
    with pytest.raises(ValueError):
        L.sg_apply(h, FakeBlock((n, P), F32), FakeBlock((n, P), F32), df64=True)
    # the level products in every arithmetic the benchmark times
    off = h.off
    for lo, li in [(l - 1, l) for l in range(1, h.p + 1)] + [(l, l - 1) for l in range(1, h.p + 1)]:
        wi, wo = off[li + 1] - off[li], off[lo + 1] - off[lo]
        for tx, ty, df in ((F32, F32, False), (F64, F64, False), (F32, F64, False), (F32, F64, True)):
            L.sg_level_apply(h, lo, li, FakeBlock((n, wi), tx), FakeBlock((n, wo), ty), FakeBlock((n, wo), tx),
                             df64=df)
            L.sg_level_apply(h, lo, li, FakeBlock((n, wi), tx), FakeBlock((n, wo), ty), df64=df)
        Yt = FakeBlock((n, wo), F64)
        L.sg_level_apply(h, lo, li, FakeBlock((n, wi), F64), Yt, Yt)      # in place
        with pytest.raises(ValueError):
            L.sg_level_apply(h, lo, li, FakeBlock((n, wi + 1), F64), FakeBlock((n, wo), F64))
        with pytest.raises(ValueError):
            L.sg_level_apply(h, lo, li, FakeBlock((n, wi), F64), FakeBlock((n, wo + 1), F64))
        with pytest.raises(ValueError):          # mixed: the output is FP32
            L.sg_level_apply(h, lo, li, FakeBlock((n, wi), F32), FakeBlock((n, wo), F64), FakeBlock((n, wo), F64))
    # levels out of range are left to the library (it answers SG_ERR_INVALID_ARG)
    L.sg_level_apply(h, 0, h.p + 3, FakeBlock((n, 5), F64), None, FakeBlock((n, 5), F64))
    assert L._lib.LIB.calls.count("sg_level_apply") == 2 * h.p * (8 + 1) + 1


def test_solves_and_preconditioners_take_n_by_P_fp64_blocks(L):
    h = _handle(L)
    n, P = h.n, h.P
    for fn in (L.hsc_precond_apply, L.bgs_precond_apply, L.mean_precond_apply):
        fn(h, FakeBlock((n, P)))
        fn(h, FakeBlock((n, P)), None, FakeBlock((n, P)))
        for R, Z in (((n, P), F32), None), (((n, P - 1), F64), None), (((n, P), F64), ((n, 1), F64)):
            with pytest.raises(ValueError):
                fn(h, FakeBlock(*R), None, None if Z is None else FakeBlock(*Z))
    L.sg_solve(h, FakeBlock((n, P)))
    L.sg_solve(h, FakeBlock((n, P)), None, FakeBlock((n, P)))
    with pytest.raises(ValueError):
        L.sg_solve(h, FakeBlock((n, P - 1)))
    with pytest.raises(ValueError):
        L.sg_solve(h, FakeBlock((n, P)), None, FakeBlock((n, P), F32))
    for fn in (L.sg_vcycle_apply, L.sg_inner_solve):
        for w in (1, 17, 300):
            fn(h, FakeBlock((n, w), F32))
            fn(h, FakeBlock((n, w), F64))
        with pytest.raises(ValueError):
            fn(h, FakeBlock((n - 1, 4), F32))
        with pytest.raises(ValueError):
            fn(h, FakeBlock((n,), F32))
    assert "sg_solve" in L._lib.LIB.calls and "sg_inner_solve" in L._lib.LIB.calls


def test_host_blocks_and_batches(L):
    h1, h2 = _handle(L), _handle(L, M=2, p=2, n=9)
    L.sg_solve_host(h1, FakeBlock((h1.n, h1.P), cuda=False))
    with pytest.raises(ValueError):
        L.sg_solve_host(h1, FakeBlock((h1.n, h1.P - 1), cuda=False))
    b = object.__new__(L.SGBatch)
    b.problems, b.b = [h1, h2], None
    Fs = [FakeBlock((h.n, h.P)) for h in (h1, h2)]
    b.solve(Fs)
    b.solve(Fs, None, [FakeBlock((h.n, h.P)) for h in (h1, h2)])
    with pytest.raises(ValueError):
        b.solve(Fs[::-1])
    with pytest.raises(ValueError):
        b.solve(Fs[:1])
    with pytest.raises(ValueError):
        b.solve(Fs, None, Fs[:1])
    Fh = [FakeBlock((h.n, h.P), cuda=False) for h in (h1, h2)]
    b.solve_host(Fh, None, [FakeBlock((h.n, h.P), cuda=False) for h in (h1, h2)])
    with pytest.raises(ValueError):
        b.solve_host(Fh[::-1], None, Fh[::-1])
    assert L._lib.LIB.calls.count("sg_batch_solve") == 2 and "sg_batch_solve_host" in L._lib.LIB.calls


def test_gradient_and_scales_follow_the_value_terms(L):
    h = _handle(L)
    n, P = h.n, h.P
    U, Lam = FakeBlock((n, P)), FakeBlock((n, P))
    L.sg_qoi(h, U)
    L.sg_qoi_grad(h, U, Lam, np.ones((3, h.M + 1)))
    L.sg_kl_qoi_grad(h, U, Lam, np.ones(h.M + 2))
    L.sg_set_scales(h, np.ones(h.M + 1))
    for bad in (np.ones((3, h.M)), np.ones(h.M + 1), np.ones((0, h.M + 1))):
        with pytest.raises(ValueError):
            L.sg_qoi_grad(h, U, Lam, bad)
    with pytest.raises(ValueError):
        L.sg_qoi(h, FakeBlock((n, P - 1)))
    with pytest.raises(ValueError):
        L.sg_kl_qoi_grad(h, U, FakeBlock((n, P), F32), np.ones(h.M + 2))
    # a gPC coefficient of degree q: one value term per coefficient polynomial
    g = _handle(L, M=2, p=2, q=4)
    assert g.nterm == 15
    L.sg_set_scales(g, np.ones(15))
    L.sg_qoi_grad(g, FakeBlock((g.n, g.P)), FakeBlock((g.n, g.P)), np.ones((2, 15)))
    with pytest.raises(ValueError):
        L.sg_set_scales(g, np.ones(g.M + 1))
    with pytest.raises(ValueError):
        L.sg_qoi_grad(g, FakeBlock((g.n, g.P)), FakeBlock((g.n, g.P)), np.ones((2, g.M + 1)))


def test_setup_arrays_are_sized_before_the_library_reads_them(L):
    """SGProblem hands the pattern, the values and the mass matrix to
    sg_setup as bare host pointers: values of the wrong term count and a mass
    array of the wrong length are refused first."""
    import sg_inputs as S
    prob = S.make_problem(4, 2, 0.3, 0.5)
    with pytest.raises(ValueError):
        L.SGProblem(4, 4, 2, 2, prob.rowptr, prob.colidx, prob.vals[:, :2], prob.mass)
    with pytest.raises(ValueError):
        L.SGProblem(4, 4, 2, 2, prob.rowptr, prob.colidx, prob.vals, prob.mass[:-1])
    assert "sg_setup" not in L._lib.LIB.calls
