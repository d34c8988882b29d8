"""Pins of the oracle's Krylov pieces: textbook CG properties, the Lanczos
estimate on a known spectrum, and the paper's own iteration counts and
condition estimates (Sec. 6, Tables 1 and 3) as soft pins."""
import math
import os

import numpy as np
import pytest

import sg_inputs as S
from oracle import chaos, hsc, krylov, sg_operator as so

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_cg_on_known_spectrum_and_lanczos_estimate():
    """CG on diag(1..m) converges in at most m steps and the Lanczos estimate
    after convergence is the exact condition number m."""
    m = 12
    d = np.arange(1, m + 1, dtype=np.float64)
    f = np.ones(m)
    x, info = krylov.fcg(lambda v: d * v, f, None, tol=1e-14, maxit=50, flexible=False)
    assert info["iters"] <= m
    assert np.allclose(x, 1.0 / d, atol=1e-12)
    assert krylov.lanczos_kappa(info["alpha"], info["beta"]) == pytest.approx(m, rel=1e-8)


def test_exact_preconditioner_converges_in_one_step():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((20, 20))
    A = X @ X.T + 20 * np.eye(20)
    f = rng.standard_normal(20)
    Ainv = np.linalg.inv(A)
    for flexible in (True, False):
        x, info = krylov.fcg(lambda v: A @ v, f, lambda r: Ainv @ r, tol=1e-12, flexible=flexible)
        assert info["iters"] == 1
        assert np.allclose(A @ x, f, atol=1e-10)


def test_fcg_sg_solution_matches_direct_solve():
    prob = S.make_problem(8, 2, 0.3, 0.5)
    M, p = 2, 3
    A = so.kl_matrices(prob.rowptr, prob.colidx, prob.vals)
    G = chaos.g_matrices(M, p)
    _, off = chaos.multi_indices(M, p)
    F = S.make_rhs(prob, p)
    U_ref = so.direct_solve(A, G, F)
    ap = lambda U: so.sg_apply(A, G, U)
    for prec in (None, lambda R: hsc.hsc_apply(A, G, off, R), lambda R: hsc.mean_apply(A, R)):
        U, info = krylov.fcg(ap, F, prec, tol=1e-13, maxit=2000)
        assert info["converged"]
        assert np.abs(U - U_ref).max() < 1e-10 * np.abs(U_ref).max()


def _read(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


def _paper_run(M, p, cov, ne=10):
    """Sec. 6 setting: 10x10 Q1 mesh (Table 4: ne x ne), L = 0.5, k0 = 1. The
    reading of the garbled distribution of xi (printed ``U[0,1]``) is
    ``U(-1, 1)``: in this build's unit-variance variables that is
    sigma = CoV / sqrt(3)."""
    prob = S.make_problem(ne, M, cov / math.sqrt(3.0), 0.5)
    A = so.kl_matrices(prob.rowptr, prob.colidx, prob.vals)
    G = chaos.g_matrices(M, p)
    _, off = chaos.multi_indices(M, p)
    F = S.make_rhs(prob, p)
    a0 = hsc.A0Solver(A[0])
    ap = lambda U: so.sg_apply(A, G, U)
    out = {}
    for name, prec in (("mean", lambda R: hsc.mean_apply(A, R, a0)),
                       ("hsc", lambda R: hsc.hsc_apply(A, G, off, R, a0solve=a0)),
                       ("bgs", lambda R: hsc.bgs_apply(A, G, R, dsolve=lambda j, x: a0(x[:, None])[:, 0]))):
        _, info = krylov.fcg(ap, F, prec, tol=1e-8, maxit=500)
        out[name] = (info["iters"], krylov.lanczos_kappa(info["alpha"], info["beta"]))
    return out


@pytest.mark.parametrize("row", _read("sec6_table3_vary_cov_full.txt"), ids=lambda r: f"cov{int(r[0])}")
def test_paper_table3_soft(row):
    """Iterations within 2 and kappa within 10 % of Table 3 (the paper's KL is
    a discrete eigenproblem on its mesh and its dof count includes boundary
    nodes, so equality is not expected)."""
    cov, _, _, m_it, m_k, b_it, b_k, h_it, h_k = row
    out = _paper_run(4, 4, cov / 100.0)
    _uniform_soft(out, m_it, m_k, b_it, b_k, h_it, h_k)
    # the method's claim: HSC needs fewer iterations than the mean-based one
    assert out["hsc"][0] < out["mean"][0]


@pytest.mark.parametrize("row", _read("sec6_table1_vary_N_full.txt"), ids=lambda r: f"N{int(r[0])}")
def test_paper_table1_soft(row):
    N, _, _, _, m_it, m_k, b_it, b_k, h_it, h_k = row
    _uniform_soft(_paper_run(int(N), 4, 0.5), m_it, m_k, b_it, b_k, h_it, h_k)


def _uniform_soft(out, m_it, m_k, b_it, b_k, h_it, h_k):
    assert abs(out["mean"][0] - m_it) <= 2
    assert abs(out["bgs"][0] - b_it) <= 2
    assert abs(out["hsc"][0] - h_it) <= 2
    assert out["mean"][1] == pytest.approx(m_k, rel=0.10)
    assert out["bgs"][1] == pytest.approx(b_k, rel=0.10)
    assert out["hsc"][1] == pytest.approx(h_k, rel=0.10)


@pytest.mark.parametrize("row", _read("sec6_table2_vary_P.txt"),
                         ids=lambda r: f"p{int(r[0])}")
def test_paper_table2_soft(row):
    """Table 2 (N = 4, CoV 50 %, chaos degree varied), same soft bounds as
    Tables 1 and 3."""
    p, _, _, _, m_it, m_k, b_it, b_k, h_it, h_k = row
    _uniform_soft(_paper_run(4, int(p), 0.5), m_it, m_k, b_it, b_k, h_it, h_k)


@pytest.mark.parametrize("row", _read("sec6_table4_vary_h.txt"),
                         ids=lambda r: f"h1_{int(r[0])}")
def test_paper_table4_soft(row):
    """Table 4 (N = p = 4, CoV 50 %, mesh 1/h x 1/h varied): the counts do not
    grow with the mesh, within the same soft bounds."""
    inv_h, _, _, _, m_it, m_k, b_it, b_k, h_it, h_k = row
    _uniform_soft(_paper_run(4, 4, 0.5, ne=int(inv_h)), m_it, m_k, b_it, b_k, h_it, h_k)


def test_pcg_columns_conventions():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((15, 15))
    A = X @ X.T + 15 * np.eye(15)
    Ainv = np.linalg.inv(A)
    B = rng.standard_normal((15, 4))
    B[:, 2] = 0.0
    Xs, it = krylov.pcg_columns(lambda v: A @ v, B, lambda r: Ainv @ r, tol=1e-10, maxit=30)
    assert list(it) == [1, 1, 0, 1]               # exact M0: one step; zero column done at entry
    assert np.allclose(A @ Xs, B, atol=1e-10)
    # unpreconditioned, fixed iteration count runs exactly that many steps
    Xs, it = krylov.pcg_columns(lambda v: A @ v, B, lambda r: r.copy(), tol=0.0, maxit=30, fixed_iters=3)
    assert list(it) == [3, 3, 0, 3]
    # tolerance test per column: residual below tol * ||b||
    Xs, it = krylov.pcg_columns(lambda v: A @ v, B, lambda r: r.copy(), tol=1e-3, maxit=100)
    for s in (0, 1, 3):
        assert np.linalg.norm(B[:, s] - A @ Xs[:, s]) <= 1e-3 * np.linalg.norm(B[:, s]) * (1 + 1e-9)


def _lognormal_run(M, p, cov, ne=10):
    """Sec. 6 lognormal setting: 10x10 mesh, L = 0.5, gPC expansion of the
    coefficient to degree 2p (Hermite chaos), exact inner solves; D_l is not
    block diagonal, so Algorithm 1 factors each D_l as it stands."""
    prob = S.make_lognormal_problem(ne, M, cov, 0.5, 2 * p)
    A = so.kl_matrices(prob.rowptr, prob.colidx, prob.vals)
    G = chaos.gpc_g_matrices(M, p, 2 * p)
    _, off = chaos.multi_indices(M, p)
    F = S.make_rhs(prob, p)
    a0 = hsc.A0Solver(A[0])
    ap = lambda U: so.sg_apply(A, G, U)
    out = {}
    for name, prec in (("mean", lambda R: hsc.mean_apply(A, R, a0)),
                       ("hsc", lambda R: hsc.hsc_apply(A, G, off, R, general=True, a0solve=a0)),
                       ("bgs", lambda R: hsc.bgs_apply(A, G, R))):
        _, info = krylov.fcg(ap, F, prec, tol=1e-8, maxit=1000)
        out[name] = (info["iters"], krylov.lanczos_kappa(info["alpha"], info["beta"]))
    return out


def lognormal_soft(out, m_it, m_k, b_it, b_k, h_it, h_k):
    """Soft agreement with the paper's lognormal tables: its field came from a
    discretised KL eigenproblem and its CoV reading is not stated, so the
    values agree to within 25 % in kappa and 25 % (at least 3) in
    iterations; the paper's findings hold exactly: M_HS has the smallest
    condition estimate, needs at most one iteration more than M_bGS, and both
    need far fewer than M_m."""
    for (it, k), (pit, pk) in ((out["mean"], (m_it, m_k)), (out["bgs"], (b_it, b_k)), (out["hsc"], (h_it, h_k))):
        assert abs(it - pit) <= max(3, 0.25 * pit)
        assert k == pytest.approx(pk, rel=0.25)
    assert out["hsc"][1] < out["bgs"][1] < out["mean"][1]
    assert out["hsc"][0] <= out["bgs"][0] + 1
    assert 2 * max(out["hsc"][0], out["bgs"][0]) < out["mean"][0] + 2


@pytest.mark.parametrize("row", [r for r in _read("sec6_table6_lognormal_vary_N.txt") if r[0] <= 2],
                         ids=lambda r: f"N{int(r[0])}")
def test_paper_table6_lognormal_soft(row):
    N, _, _, _, m_it, m_k, b_it, b_k, h_it, h_k = row
    lognormal_soft(_lognormal_run(int(N), 4, 1.0), m_it, m_k, b_it, b_k, h_it, h_k)


@pytest.mark.parametrize("row", [r for r in _read("sec6_table7_lognormal_vary_P.txt") if r[0] <= 3],
                         ids=lambda r: f"P{int(r[0])}")
def test_paper_table7_lognormal_soft(row):
    p, _, _, _, m_it, m_k, b_it, b_k, h_it, h_k = row
    lognormal_soft(_lognormal_run(4, int(p), 1.0), m_it, m_k, b_it, b_k, h_it, h_k)


def test_flexible_cg_keeps_consecutive_directions_conjugate():
    """Flexible CG (Sec. 5, for a preconditioner that changes from one
    application to the next): the flexible beta z_{k+1}^T (r_{k+1} - r_k) /
    rho_k is the one that makes each new search direction A-conjugate to the
    previous one, p_{k+1}^T A p_k = 0, whatever the preconditioner did; the
    standard beta rho_{k+1} / rho_k does not under a changing preconditioner.
    The search directions are the operator's inputs, recorded as it is called."""
    m = 30
    rng = np.random.default_rng(3)
    X = rng.standard_normal((m, m))
    A = X @ X.T / m + np.eye(m)
    f = rng.standard_normal(m)

    def run(flexible):
        dirs, prng = [], np.random.default_rng(8)

        def apply_A(v):
            dirs.append(v.copy())
            return A @ v

        def apply_M(r):                                # a different SPD operator at every call
            Y = prng.standard_normal((m, m))
            return (Y @ Y.T / m + 0.5 * np.eye(m)) @ r

        x, info = krylov.fcg(apply_A, f, apply_M, tol=1e-12, maxit=12, flexible=flexible)
        cos = [abs(a @ A @ b) / np.sqrt((a @ A @ a) * (b @ A @ b)) for a, b in zip(dirs[1:], dirs[:-1])]
        return x, info, cos

    x, info, cos = run(True)
    assert len(cos) >= 8 and max(cos) < 1e-10
    # the recursively updated residual is the true one
    assert info["res"][-1] == pytest.approx(np.linalg.norm(f - A @ x) / np.linalg.norm(f), rel=1e-6)
    _, _, cos_std = run(False)
    assert max(cos_std) > 1e-3


def test_pcg_iterates_minimise_the_energy_error_over_the_krylov_space():
    """Brute force of what k steps of preconditioned CG from zero compute: the
    x in span{M b, (M A) M b, ..., (M A)^{k-1} M b} that minimises the A-norm
    of the error, i.e. the Galerkin solution x = V y with V^T A V y = V^T b
    for a basis V of that space. Checked for the inner column PCG with a fixed
    iteration count and for the outer CG (standard and flexible, which coincide
    for a fixed preconditioner), with an SPD preconditioner that is neither the
    identity nor A^{-1}."""
    m = 24
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
    A = (Q * np.linspace(1.0, 40.0, m)) @ Q.T
    Y = rng.standard_normal((m, m))
    Mp = Y @ Y.T / m + 0.3 * np.eye(m)
    b = rng.standard_normal(m)
    for k in range(1, 7):
        cols = [Mp @ b]
        for _ in range(k - 1):
            cols.append(Mp @ (A @ cols[-1]))
        V, _ = np.linalg.qr(np.array(cols).T)
        x_ref = V @ np.linalg.solve(V.T @ A @ V, V.T @ b)
        scale = np.abs(x_ref).max()
        X, it = krylov.pcg_columns(lambda v: A @ v, b[:, None], lambda r: Mp @ r, tol=0.0, maxit=k, fixed_iters=k)
        assert it[0] == k
        assert np.abs(X[:, 0] - x_ref).max() <= 1e-9 * scale, k
        for flexible in (False, True):
            x, info = krylov.fcg(lambda v: A @ v, b, lambda r: Mp @ r, tol=0.0, maxit=k, flexible=flexible)
            assert info["iters"] == k
            assert np.abs(x - x_ref).max() <= 1e-9 * scale, (k, flexible)


def test_fcg_initial_guess_zero_right_hand_side_and_breakdown():
    """The edges of the outer CG: a zero right-hand side is solved at entry
    (x = 0, no iteration); an initial guess starts from r = f - A x0 (the exact
    solution needs no iteration, a perturbed one converges to the same x); a
    direction with p^T A p <= 0 (an indefinite operator) stops the iteration
    with the breakdown flag; no CG step gives the condition estimate 1."""
    rng = np.random.default_rng(6)
    X = rng.standard_normal((10, 10))
    A = X @ X.T + 10 * np.eye(10)
    f = rng.standard_normal(10)
    x, info = krylov.fcg(lambda v: A @ v, np.zeros(10), None, tol=1e-10)
    assert info["converged"] and info["iters"] == 0 and not np.any(x)
    xs = np.linalg.solve(A, f)
    x, info = krylov.fcg(lambda v: A @ v, f, None, tol=1e-10, x0=xs)
    assert info["converged"] and info["iters"] == 0 and info["res"][0] < 1e-12
    x0 = xs + 0.1 * rng.standard_normal(10)
    x, info = krylov.fcg(lambda v: A @ v, f, None, tol=1e-12, x0=x0)
    assert info["res"][0] == pytest.approx(np.linalg.norm(f - A @ x0) / np.linalg.norm(f), rel=1e-12)
    assert info["converged"] and np.abs(x - xs).max() < 1e-10 * np.abs(xs).max()
    x, info = krylov.fcg(lambda v: np.array([1.0, -2.0]) * v, np.array([1.0, 1.0]), None, tol=1e-10)
    assert info.get("breakdown") and not info["converged"] and info["iters"] == 0
    assert krylov.lanczos_kappa([], []) == 1.0
