"""The cluster-resident inner solver (one launch per batched inner PCG, the
multigrid hierarchy in the shared memory of 8-block clusters) against the
FP64 oracle and against the stand-alone kernels, on seeded inputs: fixed
iteration counts element by element, tolerance-driven solves by their true
residuals and iteration counts, Algorithm 1 and the outer solve."""
import os

import numpy as np
import pytest

import sg_inputs as S
from oracle import gmg, hsc, krylov, sg_operator as so
from tests.gpu_common import problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1205_1864_gb300 as L
    return L


def _t(x, dtype=None):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype or torch.float64, device="cuda")


def _np(t):
    return t.double().cpu().numpy()


def _pair(lib, prob, p):
    """(handle on the cluster solver, handle on the stand-alone kernels)."""
    h1 = lib.SGProblem.from_inputs(prob, p)
    os.environ["SGHSC_NO_CLUSTER"] = "1"
    try:
        h0 = lib.SGProblem.from_inputs(prob, p)
    finally:
        del os.environ["SGHSC_NO_CLUSTER"]
    return h1, h0


@pytest.mark.parametrize("ne", [16, 32, 64, 128])
def test_cluster_solver_selected(lib, ne):
    prob, A, G, off = problem(ne, 2, 1)
    h1, h0 = _pair(lib, prob, 1)
    assert h1.inner_cluster and not h0.inner_cluster


@pytest.mark.parametrize("ne,w,nu,omega", [(16, 7, 2, 0.8), (32, 13, 1, 0.8), (64, 9, 3, 0.7), (128, 37, 2, 0.8)])
def test_cluster_fixed_iterations_parity(lib, ne, w, nu, omega):
    """Three V-cycle-preconditioned CG steps per column (nu sweeps, weight
    omega) against the column-wise oracle; a zero column stays zero; the
    padded columns of the last group (w not a multiple of 4) are not written."""
    import torch
    prob, A, G, off = problem(ne, 2, 1)
    h = lib.SGProblem.from_inputs(prob, 1)
    assert h.inner_cluster
    lv = gmg.hierarchy(A[0], ne)
    B = S.random_block(prob.n, w, seed=21 + ne).astype(np.float32).astype(np.float64)
    B[:, 2] = 0.0
    o = lib.prec_opts(inner_fixed_iters=3, nu=nu, omega=omega)
    X, it = lib.sg_inner_solve(h, _t(B, torch.float32), o)
    ref, it_ref = krylov.pcg_columns(lambda v: A[0] @ v, B, lambda r: gmg.vcycle(lv, r, nu=nu, omega=omega),
                                     tol=0.0, maxit=3, fixed_iters=3)
    assert list(it) == list(it_ref)
    X = _np(X)
    scale = np.abs(ref).max(axis=0, keepdims=True) + 1e-300
    assert np.all(np.abs(X - ref) <= 1e-4 * scale)
    assert np.all(X[:, 2] == 0.0)


@pytest.mark.parametrize("ne,w", [(32, 5), (64, 11), (128, 1), (128, 21)])
def test_cluster16_fixed_iterations_parity(lib, ne, w):
    """Clusters of 16 CTAs (half the rows of every strip grid per CTA, one
    more grid on CTA 0 alone) against the column-wise oracle, and against
    clusters of 8 within FP32 rounding (the cluster sums add 16 block sums
    instead of 8)."""
    import torch
    prob, A, G, off = problem(ne, 2, 1)
    h16 = lib.SGProblem.from_inputs(prob, 1)
    if h16.inner_path(w) != 3:
        pytest.skip("clusters of 16 CTAs are not resident on this device")
    os.environ["SGHSC_NO_CLUSTER16"] = "1"
    try:
        h8 = lib.SGProblem.from_inputs(prob, 1)
    finally:
        del os.environ["SGHSC_NO_CLUSTER16"]
    assert h8.inner_path(w) == 1
    lv = gmg.hierarchy(A[0], ne)
    B = S.random_block(prob.n, w, seed=51 + ne + w).astype(np.float32).astype(np.float64)
    if w > 2:
        B[:, 2] = 0.0
    o = lib.prec_opts(inner_fixed_iters=3)
    X16, it16 = lib.sg_inner_solve(h16, _t(B, torch.float32), o)
    X8, it8 = lib.sg_inner_solve(h8, _t(B, torch.float32), o)
    ref, it_ref = krylov.pcg_columns(lambda v: A[0] @ v, B, lambda r: gmg.vcycle(lv, r), tol=0.0, maxit=3,
                                     fixed_iters=3)
    assert list(it16) == list(it_ref) and list(it8) == list(it_ref)
    X16, X8 = _np(X16), _np(X8)
    scale = np.abs(ref).max(axis=0, keepdims=True) + 1e-300
    assert np.all(np.abs(X16 - ref) <= 1e-4 * scale)
    assert np.all(np.abs(X16 - X8) <= 1e-5 * scale)
    if w > 2:
        assert np.all(X16[:, 2] == 0.0)


@pytest.mark.parametrize("tol", [1e-2, 1e-4])
def test_cluster_tolerance_matches_stand_alone(lib, tol):
    """Degree-level widths of the 128x128, M=6 workload: every column reaches
    its tolerance (true residual, FP64), and the iteration counts of the two
    solvers agree to within one (FP32 rounding can move a column across the
    threshold)."""
    import torch
    prob, A, G, off = problem(128, 2, 1)
    h1, h0 = _pair(lib, prob, 1)
    for w, seed in [(1, 31), (6, 32), (21, 33), (56, 34)]:
        B = S.random_block(prob.n, w, seed=seed)
        B[:, ::5] *= 1e-3
        o = lib.prec_opts(inner_tol=tol)
        X1, it1 = lib.sg_inner_solve(h1, _t(B, torch.float32), o)
        X0, it0 = lib.sg_inner_solve(h0, _t(B, torch.float32), o)
        X1 = _np(X1)
        B32 = B.astype(np.float32).astype(np.float64)
        res = np.linalg.norm(B32 - A[0] @ X1, axis=0) / np.linalg.norm(B32, axis=0)
        assert np.all(res <= 2 * tol), (w, res.max())
        assert np.all(np.abs(np.asarray(it1) - np.asarray(it0)) <= 1), (w, it1, it0)
        assert np.all(np.asarray(it1) >= 1)


def test_cluster_maxit_caps_every_column(lib):
    """inner_maxit ends every unfinished column after that many iterations (a
    capped inner loop is not an error); both solvers give the same iterate up
    to FP32 rounding."""
    import torch
    prob, A, G, off = problem(64, 2, 1)
    h1, h0 = _pair(lib, prob, 1)
    B = S.random_block(prob.n, 10, seed=41)
    o = lib.prec_opts(inner_tol=1e-12, inner_maxit=2)
    X1, it1 = lib.sg_inner_solve(h1, _t(B, torch.float32), o)
    X0, it0 = lib.sg_inner_solve(h0, _t(B, torch.float32), o)
    assert list(it1) == [2] * 10 and list(it0) == [2] * 10
    X1, X0 = _np(X1), _np(X0)
    assert np.abs(X1 - X0).max() <= 1e-5 * np.abs(X0).max()


def test_cluster_hsc_matches_oracle_and_stand_alone(lib):
    """Algorithm 1 with FP32 inner solves of fixed length: oracle within the
    mixed-precision bound; the two inner solvers within FP32 rounding."""
    prob, A, G, off = problem(32, 3, 3)
    h1, h0 = _pair(lib, prob, 3)
    lv = gmg.hierarchy(A[0], 32)
    R = S.random_block(prob.n, h1.P, seed=42)
    o = lib.prec_opts(precision=lib.SG_F32, inner_fixed_iters=4)
    Z1 = _np(lib.hsc_precond_apply(h1, _t(R), o))
    Z0 = _np(lib.hsc_precond_apply(h0, _t(R), o))

    def dsolve(l, X):
        return krylov.pcg_columns(lambda v: A[0] @ v, X, lambda r: gmg.vcycle(lv, r), tol=0.0, maxit=4,
                                  fixed_iters=4)[0]
    ref = hsc.hsc_apply(A, G, off, R, dsolve=dsolve)
    assert np.abs(Z1 - ref).max() <= 2e-5 * np.abs(ref).max()
    assert np.abs(Z1 - Z0).max() <= 2e-5 * np.abs(ref).max()


def test_cluster_solve_to_1e8_matches_direct(lib):
    """The mixed-precision HSC-FCG solve on the cluster solver reaches the
    relative residual 1e-8 and matches the oracle's direct solve."""
    prob, A, G, off = problem(16, 3, 3, 0.2, 0.5)
    h1, h0 = _pair(lib, prob, 3)
    F = S.make_rhs(prob, 3)
    ref = so.direct_solve(A, G, F)
    o = lib.solve_opts(lib.prec_opts(precision=lib.SG_F32), precond=lib.SG_PREC_HSC, tol=1e-8)
    U1, s1 = lib.sg_solve(h1, _t(F), o)
    U0, s0 = lib.sg_solve(h0, _t(F), o)
    assert s1.true_rel_res <= 1e-8 * 1.01
    assert np.abs(_np(U1) - ref).max() <= 1e-6 * np.abs(ref).max()
    assert abs(s1.iterations - s0.iterations) <= 1
    assert s1.inner_iters_total > 0 and s1.inner_iters_max >= 1


@pytest.mark.parametrize("nu,omega", [(1, 0.8), (3, 0.7)])
def test_wide_cluster_solver_smoothing_variants(lib, nu, omega):
    """The wide solver with one and three smoothing sweeps (other weights):
    fixed iteration counts against the oracle."""
    import torch
    prob, A, G, off = problem(128, 2, 1)
    h = lib.SGProblem.from_inputs(prob, 1)
    w = 90
    if h.inner_path(w) != 2:
        pytest.skip("the device holds too few clusters for the wide solver")
    lv = gmg.hierarchy(A[0], 128)
    B = S.random_block(prob.n, w, seed=80 + nu).astype(np.float32).astype(np.float64)
    o = lib.prec_opts(inner_fixed_iters=2, nu=nu, omega=omega)
    X, it = lib.sg_inner_solve(h, _t(B, torch.float32), o)
    ref, it_ref = krylov.pcg_columns(lambda v: A[0] @ v, B, lambda r: gmg.vcycle(lv, r, nu=nu, omega=omega),
                                     tol=0.0, maxit=2, fixed_iters=2)
    assert list(it) == list(it_ref)
    scale = np.abs(ref).max(axis=0, keepdims=True) + 1e-300
    assert np.all(np.abs(_np(X) - ref) <= 1e-4 * scale)


def test_hsc_top_level_on_wide_solver(lib):
    """Algorithm 1 on the 128x128, M=6, p=4 workload (126-column top level on
    the wide solver, its FP64-residual input variant in the pre-loop): the
    mixed-precision application against the stand-alone kernels, and the
    solve to 1e-8."""
    prob, A, G, off = problem(128, 6, 4, 0.3, 1.0)
    h1, h0 = _pair(lib, prob, 4)
    if h1.inner_path(126) != 2:
        pytest.skip("the device holds too few clusters for the wide solver")
    R = S.random_block(prob.n, h1.P, seed=90)
    o = lib.prec_opts(precision=lib.SG_F32, inner_fixed_iters=2)
    Z1 = _np(lib.hsc_precond_apply(h1, _t(R), o))
    Z0 = _np(lib.hsc_precond_apply(h0, _t(R), o))
    assert np.abs(Z1 - Z0).max() <= 1e-4 * np.abs(Z0).max()
    F = S.make_rhs(prob, 4)
    U, st = lib.sg_solve(h1, _t(F), lib.solve_opts(lib.prec_opts(precision=lib.SG_F32), precond=lib.SG_PREC_HSC,
                                                   tol=1e-8))
    assert st.true_rel_res <= 1e-8 * 1.01 and st.iterations <= 10


def test_wide_cluster_solver_parity(lib):
    """The 126-column top level of the 128x128, M=6 workload: more clusters
    than the on-chip solver keeps resident, so it takes the solver with the
    finest grid in global memory (path 2) where the device holds its clusters.
    Fixed iteration counts against the oracle and the stand-alone kernels; a
    tolerance-driven solve by its true residuals."""
    import torch
    prob, A, G, off = problem(128, 2, 1)
    h1, h0 = _pair(lib, prob, 1)
    w = 126
    path = h1.inner_path(w)
    assert path in (0, 2)
    if path == 0:
        pytest.skip("the device holds too few clusters for the wide solver")
    lv = gmg.hierarchy(A[0], 128)
    B = S.random_block(prob.n, w, seed=71).astype(np.float32).astype(np.float64)
    B[:, 9] = 0.0
    o = lib.prec_opts(inner_fixed_iters=3)
    X1, it1 = lib.sg_inner_solve(h1, _t(B, torch.float32), o)
    ref, it_ref = krylov.pcg_columns(lambda v: A[0] @ v, B, lambda r: gmg.vcycle(lv, r), tol=0.0, maxit=3,
                                     fixed_iters=3)
    assert list(it1) == list(it_ref)
    X1 = _np(X1)
    scale = np.abs(ref).max(axis=0, keepdims=True) + 1e-300
    assert np.all(np.abs(X1 - ref) <= 1e-4 * scale)
    assert np.all(X1[:, 9] == 0.0)
    X0, _ = lib.sg_inner_solve(h0, _t(B, torch.float32), o)
    assert np.all(np.abs(X1 - _np(X0)) <= 2e-5 * scale)
    Bt = S.random_block(prob.n, w, seed=72)
    Xt, itt = lib.sg_inner_solve(h1, _t(Bt, torch.float32), lib.prec_opts(inner_tol=1e-2))
    B32 = Bt.astype(np.float32).astype(np.float64)
    res = np.linalg.norm(B32 - A[0] @ _np(Xt), axis=0) / np.linalg.norm(B32, axis=0)
    assert np.all(res <= 2e-2)


def test_autotune_picks_inner_solvers(lib):
    """sg_autotune times every solver that can run each degree-level batch
    (stand-alone, 8- and 16-CTA clusters, the wide variant) and keeps one per
    width; a second handle of the same class takes the cached choice, and the
    mixed solve on the tuned handle still meets 1e-8 against the oracle."""
    from tests.gpu_common import oracle_rel_residual
    prob, A, G, off = problem(64, 4, 3, 0.2, 0.5)
    h = lib.SGProblem.from_inputs(prob, 3)
    rule = {int(off[l + 1] - off[l]): h.inner_path(int(off[l + 1] - off[l])) for l in range(4)}
    lib.sg_autotune(h)
    picks = {w: h.inner_path(w) for w in rule}
    assert all(v in (0, 1, 2, 3) for v in picks.values())
    h2 = lib.SGProblem.from_inputs(prob, 3)
    lib.sg_autotune(h2)
    assert {w: h2.inner_path(w) for w in rule} == picks
    F = S.make_rhs(prob, 3)
    o = lib.solve_opts(lib.prec_opts(precision=lib.SG_F32, df64=1), precond=lib.SG_PREC_HSC, tol=1e-8)
    U, st = lib.sg_solve(h, _t(F), o)
    assert st.status == 0
    assert oracle_rel_residual(A, G, F, _np(U)) <= 1.5e-8
