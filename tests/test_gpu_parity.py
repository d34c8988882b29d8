"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element
by element, on seeded inputs: the SG product (K1), the level products (K2),
the V-cycle (K4), the batched inner PCG (K3), Algorithm 1, the mean-based
preconditioner, the outer solve (K5) and the QoI gradient (K7)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import sg_inputs as S
from oracle import chaos, gmg, hsc, krylov, qoi, sg_operator as so
from tests.gpu_common import TOL32, TOL64, abs_bound, problem, random_csr

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


# ----------------------------------------------------------------------- tables

@pytest.mark.parametrize("M,p", [(3, 3), (6, 4), (1, 5), (10, 2)])
def test_chaos_table_matches_oracle(lib, M, p):
    prob, A, G, off = problem(4, M, p)
    h = lib.SGProblem.from_inputs(prob, p)
    alpha, loff = h.chaos_table()
    a_ref, off_ref = chaos.multi_indices(M, p)
    assert np.array_equal(alpha, a_ref)
    assert np.array_equal(loff, off_ref)
    assert h.P == math.comb(M + p, M)


# ------------------------------------------------------------------------ K1

@pytest.mark.parametrize("ne,M,p", [(16, 3, 3), (8, 2, 2), (16, 6, 4), (4, 1, 5), (32, 4, 3)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_sg_apply_parity(lib, ne, M, p, prec):
    import torch
    prob, A, G, off = problem(ne, M, p)
    h = lib.SGProblem.from_inputs(prob, p)
    U = S.random_block(prob.n, h.P, seed=1205)
    ref = so.sg_apply(A, G, U)
    bound = abs_bound(A, G, U)
    dt = torch.float64 if prec == "f64" else torch.float32
    Y = _np(lib.sg_apply(h, _t(U, dt)))
    if prec == "f32":
        # the input itself is rounded to FP32: compare with the oracle on the rounded input
        U32 = U.astype(np.float32).astype(np.float64)
        ref = so.sg_apply(A, G, U32)
    tol = TOL64 if prec == "f64" else TOL32
    assert np.all(np.abs(Y - ref) <= tol * bound + 1e-300), np.max(np.abs(Y - ref) / (bound + 1e-300))


@pytest.mark.parametrize("ne,M,p", [(16, 6, 4), (32, 4, 3)])
def test_sg_apply_pair_and_gather_forms_agree(lib, ne, M, p):
    """The pair form (one sum per distinct (k, j), shared by the couplings
    that name it) and the gather form (one sum per coupling) add the same
    terms in the same order on rows of one chunk: identical bits, FP64 and
    FP32, for the product and for a whole outer solve."""
    import os

    import torch
    prob, A, G, off = problem(ne, M, p)
    hp = lib.SGProblem.from_inputs(prob, p)
    os.environ["SGHSC_GATHER_FORM"] = "1"
    try:
        hg = lib.SGProblem.from_inputs(prob, p)
    finally:
        del os.environ["SGHSC_GATHER_FORM"]
    U = S.random_block(prob.n, hp.P, seed=77)
    for dt in (torch.float64, torch.float32):
        Yp = lib.sg_apply(hp, _t(U, dt))
        Yg = lib.sg_apply(hg, _t(U, dt))
        assert torch.equal(Yp, Yg)
    ref = so.sg_apply(A, G, U)
    assert np.all(np.abs(_np(lib.sg_apply(hp, _t(U))) - ref) <= TOL64 * abs_bound(A, G, U) + 1e-300)
    F = S.make_rhs(prob, p)
    o = lib.solve_opts(lib.prec_opts(precision=lib.SG_F32), precond=lib.SG_PREC_HSC, tol=1e-8)
    Up, sp_ = lib.sg_solve(hp, _t(F), o)
    Ug, sg_ = lib.sg_solve(hg, _t(F), o)
    assert sp_.iterations == sg_.iterations and torch.equal(Up, Ug)


def test_sg_apply_general_csr_ragged_rows(lib):
    """A random pattern with empty rows and rows longer than 9 nonzeros (no mesh)."""
    import torch
    n, M, p = 97, 3, 2
    rowptr, colidx = random_csr(n, seed=8)
    rng = np.random.default_rng(9)
    vals = rng.uniform(-1, 1, size=(len(colidx), M + 1))
    h = lib.SGProblem(0, 0, M, p, rowptr, colidx, vals)
    A = so.kl_matrices(rowptr, colidx, vals)
    G = chaos.g_matrices(M, p)
    U = S.random_block(n, h.P, seed=3)
    Y = _np(lib.sg_apply(h, _t(U)))
    ref = so.sg_apply(A, G, U)
    assert np.all(np.abs(Y - ref) <= TOL64 * abs_bound(A, G, U) + 1e-300)
    assert np.all(Y[3::7] == 0.0)      # empty rows give exact zeros


def test_sg_apply_p0_and_m0(lib):
    """Degenerate chaos spaces: p = 0 (the mean problem alone) and M = 0."""
    for M, p in ((3, 0), (0, 2)):
        prob = S.make_problem(8, max(M, 1), 0.3, 0.5)
        vals = prob.vals[:, : M + 1]
        h = lib.SGProblem(8, 8, M, p, prob.rowptr, prob.colidx, vals)
        assert h.P == 1
        A = so.kl_matrices(prob.rowptr, prob.colidx, vals)
        U = S.random_block(prob.n, 1, seed=2)
        Y = _np(lib.sg_apply(h, _t(U)))
        assert np.allclose(Y, A[0] @ U, rtol=0, atol=1e-13)


# ------------------------------------------------------------------------ K2

@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_level_apply_parity(lib, prec):
    import torch
    ne, M, p = 16, 4, 3
    prob, A, G, off = problem(ne, M, p)
    h = lib.SGProblem.from_inputs(prob, p)
    dt = torch.float64 if prec == "f64" else torch.float32
    tol = TOL64 if prec == "f64" else TOL32
    for lo, li in [(l - 1, l) for l in range(1, p + 1)] + [(l, l - 1) for l in range(1, p + 1)]:
        win, wout = off[li + 1] - off[li], off[lo + 1] - off[lo]
        X = S.random_block(prob.n, win, seed=10 + lo)
        Yin = S.random_block(prob.n, wout, seed=20 + li)
        if prec == "f32":
            X = X.astype(np.float32).astype(np.float64)
            Yin = Yin.astype(np.float32).astype(np.float64)
        Y = _np(lib.sg_level_apply(h, lo, li, _t(X, dt), _t(Yin, dt)))
        ref = Yin - so.level_apply(A, G, off, lo, li, X)
        bound = np.abs(Yin) + so.level_apply([abs(a) for a in A], [abs(g) for g in G], off, lo, li, np.abs(X))
        assert np.all(np.abs(Y - ref) <= tol * bound + 1e-300), (lo, li)


# ------------------------------------------------------------------------ K4

@pytest.mark.parametrize("ne,w,nu", [(16, 1, 2), (16, 7, 2), (32, 33, 2), (8, 300, 2), (64, 5, 2), (128, 40, 2),
                                     (64, 9, 1), (64, 3, 3), (128, 1, 2), (64, 513, 2)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_vcycle_parity(lib, ne, w, nu, prec):
    import torch
    prob, A, G, off = problem(ne, 2, 1)
    h = lib.SGProblem.from_inputs(prob, 1)
    lv = gmg.hierarchy(A[0], ne)
    B = S.random_block(prob.n, w, seed=ne + w)
    dt = torch.float64 if prec == "f64" else torch.float32
    if prec == "f32":
        B = B.astype(np.float32).astype(np.float64)
    o = lib.prec_opts(nu=nu, omega=0.8)
    X = _np(lib.sg_vcycle_apply(h, _t(B, dt), o))
    ref = gmg.vcycle(lv, B, nu=nu, omega=0.8)
    scale = np.abs(ref).max(axis=0, keepdims=True)
    tol = 1e-12 if prec == "f64" else 2e-5
    assert np.all(np.abs(X - ref) <= tol * scale)


# ------------------------------------------------------------------------ K3

@pytest.mark.parametrize("ne,w", [(32, 13), (64, 13), (128, 300)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_inner_pcg_fixed_iterations_parity(lib, prec, ne, w):
    """Same iteration count on both sides: the batched CG with V-cycle equals
    the column-wise oracle up to rounding."""
    import torch
    prob, A, G, off = problem(ne, 2, 1)
    h = lib.SGProblem.from_inputs(prob, 1)
    lv = gmg.hierarchy(A[0], ne)
    B = S.random_block(prob.n, w, seed=5)
    B[:, 4] = 0.0                                     # a zero column is done at entry
    dt = torch.float64 if prec == "f64" else torch.float32
    if prec == "f32":
        B = B.astype(np.float32).astype(np.float64)
    o = lib.prec_opts(inner_fixed_iters=3)
    X, it = lib.sg_inner_solve(h, _t(B, dt), o)
    ref, it_ref = krylov.pcg_columns(lambda v: A[0] @ v, B, lambda r: gmg.vcycle(lv, r), tol=0.0, maxit=3,
                                     fixed_iters=3)
    assert list(it) == list(it_ref)
    X = _np(X)
    scale = np.abs(ref).max(axis=0, keepdims=True) + 1e-300
    tol = 1e-11 if prec == "f64" else 1e-4
    assert np.all(np.abs(X - ref) <= tol * scale)
    assert np.all(X[:, 4] == 0.0)


def test_repeated_solves_are_bitwise_identical_and_graphs_reused(lib):
    """Fixed-order reductions: the same solve twice gives the same bits; a
    change of options builds a second graph and does not disturb the first."""
    prob, A, G, off = problem(64, 3, 3)
    h = lib.SGProblem.from_inputs(prob, 3)
    F = _t(S.make_rhs(prob, 3))
    o1 = lib.solve_opts(lib.prec_opts(precision=lib.SG_F32), precond=lib.SG_PREC_HSC, tol=1e-10)
    o2 = lib.solve_opts(lib.prec_opts(precision=lib.SG_F64), precond=lib.SG_PREC_MEAN, tol=1e-10)
    U1, s1 = lib.sg_solve(h, F, o1)
    U1 = U1.clone()
    U2, s2 = lib.sg_solve(h, F, o2)
    U3, s3 = lib.sg_solve(h, F, o1)
    assert s1.iterations == s3.iterations
    assert bool((U1 == U3).all())
    assert np.abs(_np(U1) - _np(U2)).max() <= 1e-8 * np.abs(_np(U2)).max()


@pytest.mark.parametrize("tol", [1e-2, 1e-6])
def test_inner_pcg_tolerance_per_column(lib, tol):
    import torch
    ne, w = 64, 40
    prob, A, G, off = problem(ne, 2, 1)
    h = lib.SGProblem.from_inputs(prob, 1)
    B = S.random_block(prob.n, w, seed=6)
    B[:, ::5] *= 1e-3                                 # uneven column scales
    X, it = lib.sg_inner_solve(h, _t(B), lib.prec_opts(precision=lib.SG_F64, inner_tol=tol))
    X = _np(X)
    res = np.linalg.norm(B - A[0] @ X, axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(res <= tol * (1 + 1e-6))
    assert np.all(it >= 1)


# ----------------------------------------------------------------- Algorithm 1

def _oracle_inner(A, lv, fixed):
    def dsolve(l, X):
        return krylov.pcg_columns(lambda v: A[0] @ v, X, lambda r: gmg.vcycle(lv, r), tol=0.0, maxit=fixed,
                                  fixed_iters=fixed)[0]
    return dsolve


@pytest.mark.parametrize("ne,M,p", [(16, 3, 3), (8, 2, 4), (16, 1, 2)])
def test_hsc_fp64_matches_oracle_with_same_inner_solver(lib, ne, M, p):
    """Algorithm 1 on the GPU (FP64) against the oracle's Algorithm 1 with the
    identical inner solver (fixed count of V-cycle-preconditioned CG steps)."""
    prob, A, G, off = problem(ne, M, p)
    h = lib.SGProblem.from_inputs(prob, p)
    lv = gmg.hierarchy(A[0], ne)
    R = S.random_block(prob.n, h.P, seed=7)
    o = lib.prec_opts(precision=lib.SG_F64, inner_fixed_iters=4)
    Z = _np(lib.hsc_precond_apply(h, _t(R), o))
    ref = hsc.hsc_apply(A, G, off, R, dsolve=_oracle_inner(A, lv, 4))
    assert np.abs(Z - ref).max() <= 1e-10 * np.abs(ref).max()


def test_hsc_tight_inner_matches_exact_algorithm1(lib):
    prob, A, G, off = problem(16, 3, 3)
    h = lib.SGProblem.from_inputs(prob, 3)
    R = S.random_block(prob.n, h.P, seed=8)
    Z = _np(lib.hsc_precond_apply(h, _t(R), lib.prec_opts(precision=lib.SG_F64, inner_tol=1e-13)))
    ref = hsc.hsc_apply(A, G, off, R)
    assert np.abs(Z - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("top64", [0, 1])
def test_hsc_mixed_precision_matches_oracle(lib, top64):
    prob, A, G, off = problem(16, 3, 3)
    h = lib.SGProblem.from_inputs(prob, 3)
    lv = gmg.hierarchy(A[0], 16)
    R = S.random_block(prob.n, h.P, seed=9)
    o = lib.prec_opts(precision=lib.SG_F32, top_level_f64=top64, inner_fixed_iters=4)
    Z = _np(lib.hsc_precond_apply(h, _t(R), o))
    ref = hsc.hsc_apply(A, G, off, R, dsolve=_oracle_inner(A, lv, 4))
    assert np.abs(Z - ref).max() <= 2e-5 * np.abs(ref).max()


def test_mean_preconditioner_parity(lib):
    prob, A, G, off = problem(16, 3, 3)
    h = lib.SGProblem.from_inputs(prob, 3)
    R = S.random_block(prob.n, h.P, seed=10)
    Z = _np(lib.mean_precond_apply(h, _t(R), lib.prec_opts(precision=lib.SG_F64, inner_tol=1e-13)))
    ref = hsc.mean_apply(A, R)
    assert np.abs(Z - ref).max() <= 1e-10 * np.abs(ref).max()


def test_hsc_zero_rhs_and_first_iteration_sparsity(lib):
    """The first outer residual has only the mean column; levels >= 1 start
    with zero right-hand sides, which the inner solver finishes at entry."""
    prob, A, G, off = problem(16, 2, 3)
    h = lib.SGProblem.from_inputs(prob, 3)
    F = S.make_rhs(prob, 3)
    Z = _np(lib.hsc_precond_apply(h, _t(F), lib.prec_opts(precision=lib.SG_F64, inner_tol=1e-13)))
    ref = hsc.hsc_apply(A, G, off, F)
    assert np.abs(Z - ref).max() <= 1e-10 * np.abs(ref).max()
    Z0 = _np(lib.hsc_precond_apply(h, _t(np.zeros_like(F)), lib.prec_opts()))
    assert np.all(Z0 == 0.0)


# ------------------------------------------------------------------------ K5

def test_solve_fp64_matches_direct_solve_cfg1(lib):
    """Configuration 1 (16x16, M=3, p=3, sigma=0.2, L=0.5), all FP64: solved to
    rel.res 1e-13, within 1e-10 of the dense direct solve."""
    c = S.CONFIGS["cfg1_fp64_16x16_M3_p3"]
    prob, A, G, off = problem(c["ne"], c["M"], c["p"], c["sigma"], c["corr_len"])
    h = lib.SGProblem.from_inputs(prob, c["p"])
    F = S.make_rhs(prob, c["p"])
    K = so.global_matrix_space_major(A, G).toarray()
    ref = np.linalg.solve(K, F.ravel()).reshape(F.shape)
    o = lib.solve_opts(lib.prec_opts(precision=lib.SG_F64, inner_tol=1e-2), precond=lib.SG_PREC_HSC, tol=1e-13)
    U, st = lib.sg_solve(h, _t(F), o)
    U = _np(U)
    assert st.true_rel_res <= 1e-12
    assert np.abs(U - ref).max() <= 1e-10 * np.abs(ref).max()
    assert st.iterations < 30


def test_solve_mixed_matches_oracle(lib):
    c = S.CONFIGS["cfg1_fp64_16x16_M3_p3"]
    prob, A, G, off = problem(c["ne"], c["M"], c["p"], c["sigma"], c["corr_len"])
    h = lib.SGProblem.from_inputs(prob, c["p"])
    F = S.make_rhs(prob, c["p"])
    ref = so.direct_solve(A, G, F)
    o = lib.solve_opts(lib.prec_opts(precision=lib.SG_F32), precond=lib.SG_PREC_HSC, tol=1e-12)
    U, st = lib.sg_solve(h, _t(F), o)
    assert np.abs(_np(U) - ref).max() <= 1e-7 * np.abs(ref).max()


@pytest.mark.parametrize("precond", ["none", "mean", "hsc"])
def test_solve_1e8_and_iteration_ordering(lib, precond):
    """Stopping at 1e-8 (Sec. 6): the oracle recomputes the true residual of the
    GPU solution in FP64; HSC needs fewer iterations than mean-based."""
    prob, A, G, off = problem(32, 4, 3, sigma=0.3, corr=0.5)
    h = lib.SGProblem.from_inputs(prob, 3)
    F = S.make_rhs(prob, 3)
    kind = {"none": lib.SG_PREC_NONE, "mean": lib.SG_PREC_MEAN, "hsc": lib.SG_PREC_HSC}[precond]
    o = lib.solve_opts(lib.prec_opts(precision=lib.SG_F32), precond=kind, tol=1e-8, maxit=1000)
    U, st = lib.sg_solve(h, _t(F), o)
    U = _np(U)
    res = np.linalg.norm(F - so.sg_apply(A, G, U)) / np.linalg.norm(F)
    assert res <= 1.5e-8
    ref_it = {"none": 50, "mean": 10, "hsc": 4}[precond]
    assert st.iterations >= ref_it
    if precond == "hsc":
        _, st_m = lib.sg_solve(h, _t(F), lib.solve_opts(lib.prec_opts(precision=lib.SG_F64), precond=lib.SG_PREC_MEAN))
        assert st.iterations < st_m.iterations


def test_solve_lanczos_estimate_matches_oracle(lib):
    prob, A, G, off = problem(16, 3, 3, sigma=0.3)
    h = lib.SGProblem.from_inputs(prob, 3)
    F = S.make_rhs(prob, 3)
    U, st = lib.sg_solve(h, _t(F), lib.solve_opts(lib.prec_opts(precision=lib.SG_F64, inner_tol=1e-12),
                                                    precond=lib.SG_PREC_HSC, tol=1e-10))
    a0 = hsc.A0Solver(A[0])
    _, info = krylov.fcg(lambda X: so.sg_apply(A, G, X), F, lambda R: hsc.hsc_apply(A, G, off, R, a0solve=a0),
                         tol=1e-10)
    assert st.iterations == info["iters"]
    assert st.kappa_est == pytest.approx(krylov.lanczos_kappa(info["alpha"], info["beta"]), rel=1e-6)


# ------------------------------------------------------------------------ errors

def test_error_paths(lib):
    import torch
    prob, A, G, off = problem(16, 2, 2)
    h = lib.SGProblem.from_inputs(prob, 2)
    F = S.make_rhs(prob, 2)
    # maxit reached
    with pytest.raises(lib.SGError) as e:
        lib.sg_solve(h, _t(F), lib.solve_opts(precond=lib.SG_PREC_NONE, maxit=2))
    assert e.value.status == 6
    # non-finite right-hand side -> breakdown, no trap
    Fn = F.copy()
    Fn[3, 0] = np.nan
    with pytest.raises(lib.SGError) as e:
        lib.sg_solve(h, _t(Fn), lib.solve_opts(precond=lib.SG_PREC_NONE))
    assert e.value.status in (5, 4)
    # the handle still works afterwards
    U, st = lib.sg_solve(h, _t(F), lib.solve_opts())
    assert st.status == 0
    # malformed pattern rejected before any launch
    bad = prob.colidx.copy()
    bad[5] = prob.n + 3
    with pytest.raises(lib.SGError) as e:
        lib.SGProblem(16, 16, 2, 2, prob.rowptr, bad, prob.vals)
    assert e.value.status == 1
    # wrong mesh size
    with pytest.raises(lib.SGError):
        lib.SGProblem(8, 8, 2, 2, prob.rowptr, prob.colidx, prob.vals)


def test_indefinite_operator_reports_breakdown(lib):
    """sigma far beyond ellipticity (Sec. 6: above CoV 55% A need not be
    positive definite): the oracle finds a negative eigenvalue of the
    assembled matrix and its CG meets p^T A p <= 0; the GPU solve must stop
    with SG_ERR_BREAKDOWN, not report success, and leave the handle usable."""
    prob, A, G, off = problem(8, 2, 3, sigma=3.0)
    K = so.global_matrix_space_major(A, G).toarray()
    assert np.linalg.eigvalsh(K)[0] < 0
    F = S.make_rhs(prob, 3)
    _, info = krylov.fcg(lambda X: so.sg_apply(A, G, X), F, None, tol=1e-8, maxit=400)
    assert info.get("breakdown") and not info["converged"]
    h = lib.SGProblem.from_inputs(prob, 3)
    for precond in (lib.SG_PREC_NONE, lib.SG_PREC_MEAN, lib.SG_PREC_HSC):
        U, st = lib.sg_solve(h, _t(F), lib.solve_opts(precond=precond, maxit=400), raise_on_error=False)
        if precond == lib.SG_PREC_NONE:
            assert st.status == 5, st.status
            assert st.iterations <= info["iters"] + 1
        else:
            assert st.status in (4, 5), st.status
    prob2, A2, G2, off2 = problem(8, 2, 3, sigma=0.3)
    h2 = lib.SGProblem.from_inputs(prob2, 3)
    U, st = lib.sg_solve(h2, _t(S.make_rhs(prob2, 3)), lib.solve_opts())
    assert st.status == 0


def test_null_pointers_rejected_before_any_launch(lib):
    """Every entry point rejects a NULL handle or buffer with SG_ERR_INVALID_ARG."""
    import ctypes as C

    import torch
    from paper_1205_1864_gb300 import _lib
    prob, A, G, off = problem(8, 2, 2)
    h = lib.SGProblem.from_inputs(prob, 2)
    F = _t(S.make_rhs(prob, 2))
    U = torch.empty_like(F)
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    o = lib.solve_opts()
    st = _lib.sg_solve_stats()
    fp, up = C.c_void_p(F.data_ptr()), C.c_void_p(U.data_ptr())
    LIB = _lib.LIB
    assert LIB.sg_solve(h.h, None, up, C.byref(o), C.byref(st), s) == 1
    assert LIB.sg_solve(h.h, fp, None, C.byref(o), C.byref(st), s) == 1
    assert LIB.sg_solve(None, fp, up, C.byref(o), C.byref(st), s) == 1
    assert LIB.sg_solve(h.h, fp, up, None, C.byref(st), s) == 1
    assert LIB.sg_apply(h.h, None, up, 0, s) == 1
    assert LIB.sg_apply(None, fp, up, 0, s) == 1
    assert LIB.hsc_precond_apply(h.h, None, up, C.byref(o.prec), s) == 1
    assert LIB.mean_precond_apply(h.h, fp, None, C.byref(o.prec), s) == 1
    assert LIB.sg_level_apply(h.h, 0, 1, None, None, up, 0, s) == 1
    assert LIB.sg_vcycle_apply(h.h, None, up, 1, 0, C.byref(o.prec), s) == 1
    assert LIB.sg_inner_solve(h.h, fp, None, 1, 0, C.byref(o.prec), None, s) == 1
    assert LIB.sg_qoi(h.h, None, None, up, s) == 1
    out = C.c_void_p()
    assert LIB.sg_setup(None, 2, 2, 0, prob.n, len(prob.colidx), None, None, None, None, C.byref(out)) == 1
    assert LIB.sg_batch_create(1, None, C.byref(out)) == 1
    assert LIB.sg_autotune(None, s) == 1
    # nothing was launched by the rejected calls: the handle still solves
    U2, st2 = lib.sg_solve(h, F, lib.solve_opts())
    assert st2.status == 0


# ------------------------------------------------------------------------ K7

def test_qoi_and_gradient_parity(lib):
    ne, M, p = 16, 3, 2
    sigma, a_mean = 0.2, 1.1
    prob, A, G, off = problem(ne, M, p, sigma=sigma, a_mean=a_mean)
    h = lib.SGProblem.from_inputs(prob, p)
    Mh = sp.csr_matrix((prob.mass, prob.colidx, prob.rowptr), shape=(prob.n, prob.n))
    U = S.random_block(prob.n, h.P, seed=11)
    Lam = S.random_block(prob.n, h.P, seed=12)
    q, dq = lib.sg_qoi(h, _t(U))
    assert float(q.item()) == pytest.approx(qoi.qoi(U, Mh), rel=1e-12)
    assert np.abs(_np(dq) - 2 * (Mh @ U)).max() <= 1e-13 * np.abs(Mh @ U).max()
    W = qoi.chain_weights(a_mean, sigma, prob.sqrt_lambda)
    g, hk = lib.sg_qoi_grad(h, _t(U), _t(Lam), W)
    hk_ref = qoi.k_resolved_products(A, G, U, Lam)
    assert np.allclose(_np(hk), hk_ref, rtol=1e-12, atol=1e-12 * np.abs(hk_ref).max())
    assert np.allclose(_np(g), W @ hk_ref, rtol=1e-11, atol=1e-12 * np.abs(W @ hk_ref).max())



@pytest.mark.parametrize("pinned", [True, False])
def test_solve_host_matches_device_solve(lib, pinned):
    """sg_solve_host on host blocks (page-locked: moved by the library's
    kernels; pageable: by cudaMemcpyAsync) gives the device entry's solution
    bit for bit, with an initial guess read from the host block too; the
    result is against the dense direct solve."""
    import torch
    c = S.CONFIGS["cfg1_fp64_16x16_M3_p3"]
    prob, A, G, off = problem(c["ne"], c["M"], c["p"], c["sigma"], c["corr_len"])
    h = lib.SGProblem.from_inputs(prob, c["p"])
    F = S.make_rhs(prob, c["p"])
    o = lib.solve_opts(lib.prec_opts(precision=lib.SG_F32, df64=1), precond=lib.SG_PREC_HSC, tol=1e-12)
    Ud, sd = lib.sg_solve(h, _t(F), o)
    Fh = torch.tensor(F, dtype=torch.float64)
    Uh = torch.full_like(Fh, 7.0)
    if pinned:
        Fh, Uh = Fh.pin_memory(), Uh.pin_memory()
    Uh, sh = lib.sg_solve_host(h, Fh, o, Uh)
    assert np.array_equal(Uh.numpy(), _np(Ud)) and sh.iterations == sd.iterations
    ref = so.direct_solve(A, G, F)
    assert np.abs(Uh.numpy() - ref).max() <= 1e-7 * np.abs(ref).max()
    # initial guess from the host block: the solution itself converges at once
    o0 = lib.solve_opts(o.prec, precond=lib.SG_PREC_HSC, tol=1e-10, use_x0=1)
    U2, s2 = lib.sg_solve_host(h, Fh, o0, Uh.clone() if not pinned else Uh.clone().pin_memory())
    assert s2.iterations <= 1
    with pytest.raises(ValueError):
        lib.sg_solve_host(h, _t(F), o)
