"""Batched solves of independent SG systems (one graph launch, ``sg_batch_*``)
and the SG-product autotuner, through the C ABI, against the individual
solves and the FP64 oracle."""
import numpy as np
import pytest

import sg_inputs as S
from oracle import sg_operator as so
from tests.gpu_common import TOL64, abs_bound, problem

pytestmark = pytest.mark.gpu

# uneven mesh size (powers of two: the multigrid hierarchy), M and p; p = 1 has a single level
SYSTEMS = [(8, 2, 2), (16, 3, 3), (4, 1, 4), (16, 4, 2), (32, 2, 3), (8, 5, 1)]


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1205_1864_gb300 as L
    return L


def _t(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _np(t):
    return t.double().cpu().numpy()


@pytest.fixture(scope="module")
def systems(lib):
    out = []
    for i, (ne, M, p) in enumerate(SYSTEMS):
        prob, A, G, off = problem(ne, M, p, sigma=0.25, corr=0.6 + 0.1 * i)
        out.append(dict(prob=prob, A=A, G=G, p=p, h=lib.SGProblem.from_inputs(prob, p),
                        F=S.make_rhs(prob, p)))
    return out


def _opts(lib, tol=1e-10):
    return lib.solve_opts(lib.prec_opts(precision=lib.SG_F32), precond=lib.SG_PREC_HSC, tol=tol)


def test_batch_matches_individual_solves_and_oracle(lib, systems):
    b = lib.SGBatch([s["h"] for s in systems])
    Us, stats = b.solve([_t(s["F"]) for s in systems], _opts(lib))
    for s, U, st in zip(systems, Us, stats):
        assert st.status == 0
        ref = so.direct_solve(s["A"], s["G"], s["F"])
        assert np.abs(_np(U) - ref).max() <= 1e-7 * np.abs(ref).max()
        Ui, sti = lib.sg_solve(s["h"], _t(s["F"]), _opts(lib))
        assert sti.iterations == st.iterations
        # same kernels, launch shapes and deterministic reductions: identical bits
        assert np.array_equal(_np(U), _np(Ui))
    b.close()


def test_batch_reuses_graph_for_new_right_hand_sides(lib, systems):
    b = lib.SGBatch([s["h"] for s in systems])
    rng = np.random.default_rng(7)
    for _ in range(2):
        Fs = [s["F"] * rng.uniform(0.5, 2.0) + 1e-3 * rng.standard_normal(s["F"].shape) for s in systems]
        Us, stats = b.solve([_t(F) for F in Fs], _opts(lib, 1e-9))
        for s, F, U in zip(systems, Fs, Us):
            res = np.linalg.norm(F - so.sg_apply(s["A"], s["G"], _np(U))) / np.linalg.norm(F)
            assert res <= 1.5e-9
    b.close()


def test_batch_failure_of_one_system_leaves_the_others(lib, systems):
    b = lib.SGBatch([s["h"] for s in systems])
    Fs = [s["F"].copy() for s in systems]
    Fs[2][1, 0] = np.nan
    with pytest.raises(lib.SGError):
        b.solve([_t(F) for F in Fs], _opts(lib))
    Us, stats = b.solve([_t(F) for F in Fs], _opts(lib), raise_on_error=False)
    assert stats[2].status != 0
    for i, (s, U, st) in enumerate(zip(systems, Us, stats)):
        if i == 2:
            continue
        assert st.status == 0
        ref = so.direct_solve(s["A"], s["G"], s["F"])
        assert np.abs(_np(U) - ref).max() <= 1e-7 * np.abs(ref).max()
    # the handles still solve on their own afterwards
    U, st = lib.sg_solve(systems[2]["h"], _t(systems[2]["F"]), _opts(lib))
    assert st.status == 0
    b.close()


def test_batch_argument_errors(lib, systems):
    h = systems[0]["h"]
    with pytest.raises(lib.SGError):
        lib.SGBatch([h, h])
    b = lib.SGBatch([h])
    with pytest.raises(ValueError):
        b.solve([])
    b.close()


def test_autotune_keeps_the_product_exact(lib):
    prob, A, G, off = problem(32, 6, 3, sigma=0.3)
    h = lib.SGProblem.from_inputs(prob, 3)
    t64, t32 = lib.sg_autotune(h)
    assert t64 in (64, 128, 256, 512, 1024) and t32 in (64, 128, 256, 512, 1024)
    U = S.random_block(h.n, h.P, seed=3)
    ref = so.sg_apply(A, G, U)
    Y = _np(lib.sg_apply(h, _t(U)))
    assert np.all(np.abs(Y - ref) <= TOL64 * abs_bound(A, G, U) + 1e-300)
    F = S.make_rhs(prob, 3)
    Us, st = lib.sg_solve(h, _t(F), _opts(lib))
    # 80k unknowns: the oracle checks the FP64 residual instead of a direct solve
    res = np.linalg.norm(F - so.sg_apply(A, G, _np(Us))) / np.linalg.norm(F)
    assert res <= 1.5e-10


def test_batch_on_host_blocks_matches_device_blocks(lib, systems):
    """SGBatch.solve_host (pinned blocks moved by the library's kernels, and
    pageable ones by the copy engine) gives the device-block solve's bits."""
    import torch
    b = lib.SGBatch([s["h"] for s in systems])
    Ud, _ = b.solve([_t(s["F"]) for s in systems], _opts(lib))
    for pinned in (True, False):
        Fh = [torch.tensor(s["F"], dtype=torch.float64) for s in systems]
        Uh = [torch.empty_like(F) for F in Fh]
        if pinned:
            Fh, Uh = [F.pin_memory() for F in Fh], [U.pin_memory() for U in Uh]
        Uh, st = b.solve_host(Fh, _opts(lib), Uh)
        for a, c, s in zip(Uh, Ud, st):
            assert s.status == 0 and np.array_equal(a.numpy(), _np(c))
    b.close()
