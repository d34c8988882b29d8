"""Pins of the oracle's Algorithm 1 (Sec. 4) against the explicit block
inverse, symmetry, definiteness and the spectral statement of Theorem 1."""
import numpy as np
import pytest

import sg_inputs as S
from oracle import chaos, hsc, krylov, sg_operator as so


def _setup(ne=4, M=2, p=3, sigma=0.4, corr=0.5):
    prob = S.make_problem(ne, M, sigma, corr)
    A = so.kl_matrices(prob.rowptr, prob.colidx, prob.vals)
    G = chaos.g_matrices(M, p)
    _, off = chaos.multi_indices(M, p)
    K = so.global_matrix_chaos_major(A, G).toarray()
    return prob, A, G, off, K


def test_block_inverse_with_true_schur_is_exact_inverse():
    """eq. (block-LU)/(block-inverse): the three factors with the true Schur
    complement S = A - B D^{-1} C invert the 2x2 block matrix."""
    prob, A, G, off, K = _setup()
    n, p = prob.n, len(off) - 2
    s, e = n * off[p], n * off[p + 1]
    Minv = hsc.block_inverse(K[:s, :s], K[:s, s:e], K[s:e, :s], K[s:e, s:e])
    assert np.abs(Minv @ K - np.eye(e)).max() < 1e-12
    # a nonsymmetric block matrix as well (the paper states the general case)
    rng = np.random.default_rng(0)
    X = rng.standard_normal((9, 9)) + 9 * np.eye(9)
    Minv = hsc.block_inverse(X[:4, :4], X[:4, 4:], X[4:, :4], X[4:, 4:])
    assert np.abs(Minv @ X - np.eye(9)).max() < 1e-13


@pytest.mark.parametrize("ne,M,p", [(4, 2, 3), (4, 3, 2), (8, 1, 4)])
def test_algorithm1_equals_recursive_block_inverse(ne, M, p):
    """Algorithm 1 (two loops over levels, space-major storage) against the
    dense recursion of eq. (block-inverse) with S_{l-1} -> A_{l-1} (chaos-major)."""
    prob, A, G, off, K = _setup(ne, M, p)
    n, P = prob.n, G[0].shape[0]
    R = S.random_block(n, P, seed=21)
    Z = hsc.hsc_apply(A, G, off, R)
    Md = hsc.hsc_dense_recursive(K, n, off)
    z = (Md @ R.T.ravel()).reshape(P, n).T
    assert np.abs(Z - z).max() < 1e-12 * np.abs(z).max()
    # the general assembled D_l solve agrees with the Lemma-based column solves
    Zg = hsc.hsc_apply(A, G, off, R, general=True)
    assert np.abs(Z - Zg).max() < 1e-12 * np.abs(z).max()


def test_hsc_symmetric_positive_definite():
    """Sec. 4, Theorem 1: M_P is SPD for SPD A_P."""
    prob, A, G, off, K = _setup(4, 2, 3)
    n, P = prob.n, G[0].shape[0]
    x = S.random_block(n, P, seed=1)
    y = S.random_block(n, P, seed=2)
    Mx = hsc.hsc_apply(A, G, off, x)
    My = hsc.hsc_apply(A, G, off, y)
    assert abs(np.sum(y * Mx) - np.sum(x * My)) < 1e-12 * abs(np.sum(y * Mx))
    Md = hsc.hsc_dense_recursive(K, n, off)
    assert np.abs(Md - Md.T).max() < 1e-12 * np.abs(Md).max()
    assert np.linalg.eigvalsh(0.5 * (Md + Md.T))[0] > 0


@pytest.mark.parametrize("ne,M,p,sigma", [(4, 2, 3, 0.4), (4, 3, 2, 0.5), (8, 1, 3, 0.5)])
def test_theorem1_spectrum(ne, M, p, sigma):
    """Sec. 4, eq. (AS-ineq) and Theorem 1, with exact inner solves.

    Derivation used for the pin: A_l = L diag(S_{l-1}, D_l) L^T gives
    spec(M_l A_l) = spec(M_{l-1} S_{l-1}) U {1}; with c_{l,1} A_l <= S_l <= c_{l,2} A_l
    and c_{l,2} <= 1 (S_l = A_l - B D^{-1} B^T <= A_l) every eigenvalue of
    M_P A_P lies in [prod_l c_{l,1}, 1] and 1 is attained. The printed bound
    prod c_{l,2}/c_{l,1} omits the eigenvalue 1 of the D block; it is checked
    here against the computed kappa as well: kappa <= 1 / prod c_{l,1} holds.
    """
    prob, A, G, off, K = _setup(ne, M, p, sigma)
    n = prob.n
    Md = hsc.hsc_dense_recursive(K, n, off)
    ev = np.sort(np.linalg.eigvals(Md @ K).real)
    cs = hsc.schur_constants(K, n, off)
    c1 = np.prod([c[0] for c in cs])
    assert all(0 < a <= b <= 1 + 1e-12 for a, b in cs)
    assert ev[-1] == pytest.approx(1.0, abs=1e-10)
    assert ev[0] >= c1 * (1 - 1e-10)
    kappa = ev[-1] / ev[0]
    assert kappa <= 1.0 / c1 * (1 + 1e-10)


def test_mean_preconditioner_is_blockwise_A0_inverse():
    prob, A, G, off, K = _setup(4, 2, 2)
    n, P = prob.n, G[0].shape[0]
    R = S.random_block(n, P, seed=3)
    Z = hsc.mean_apply(A, R)
    assert np.abs(A[0] @ Z - R).max() < 1e-12


@pytest.mark.parametrize("M,p", [(2, 2), (3, 2), (1, 3)])
def test_bgs_matches_block_triangular_solves(M, p):
    """M_bGS (Sec. 6, zero initial guess) against its closed form
    (D + U)^{-1} D (D + L)^{-1} built from the dense chaos-major matrix; it is
    symmetric and positive definite, and with the linear KL expansion the
    blocks of one degree do not couple (so a level-batched sweep is the same
    sweep)."""
    prob = S.make_problem(4, M, 0.3, 0.5)
    A = so.kl_matrices(prob.rowptr, prob.colidx, prob.vals)
    G = chaos.g_matrices(M, p)
    _, off = chaos.multi_indices(M, p)
    n, P = prob.n, G[0].shape[0]
    K = so.global_matrix_chaos_major(A, G).toarray()
    Mb = hsc.bgs_dense(K, n, P)
    R = S.random_block(n, P, seed=3)
    ref = (Mb @ R.T.ravel()).reshape(P, n).T
    U = hsc.bgs_apply(A, G, R)
    assert np.abs(U - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(Mb - Mb.T).max() <= 1e-12 * np.abs(Mb).max()
    assert np.linalg.eigvalsh(0.5 * (Mb + Mb.T))[0] > 0
    for d in range(p + 1):
        for j in range(off[d], off[d + 1]):
            for l in range(off[d], off[d + 1]):
                if j != l:
                    assert all(Gk[j, l] == 0.0 for Gk in G)


@pytest.mark.parametrize("M,p", [(2, 2), (3, 3), (2, 1)])
def test_schur_reduced_solve_recovers_the_full_solution(M, p):
    """Sec. 5, eq. (global-Schur-system): with exact D_p solves the reduced
    iteration and the recovery of u^p give the solution of the full system
    (the direct solve), and the Schur complement S_{p-1} = A_{p-1} - B_p
    D_p^{-1} C_p has a condition number no larger than A's (dense, tiny)."""
    prob = S.make_problem(8, M, 0.3, 0.5)
    A = so.kl_matrices(prob.rowptr, prob.colidx, prob.vals)
    G = chaos.g_matrices(M, p)
    _, off = chaos.multi_indices(M, p)
    F = S.make_rhs(prob, p)
    F[:, -1] = S.random_block(prob.n, 1, seed=5)[:, 0]     # a nonzero degree-p part exercises g and the recovery
    U, info = hsc.schur_reduced_solve(A, G, off, F, tol=1e-13)
    ref = so.direct_solve(A, G, F)
    assert info["converged"]
    assert np.abs(U - ref).max() <= 1e-10 * np.abs(ref).max()
    n = prob.n
    K = so.global_matrix_chaos_major(A, G).toarray()
    e = n * off[p]
    Sd = K[:e, :e] - K[:e, e:] @ np.linalg.solve(K[e:, e:], K[e:, :e])
    evs, eva = np.linalg.eigvalsh(0.5 * (Sd + Sd.T)), np.linalg.eigvalsh(K)
    assert evs[-1] / evs[0] <= eva[-1] / eva[0] * (1 + 1e-12)


def test_general_prec_variants_match_the_paper_formula():
    """Sec. 5, eq. (general-prec): Algorithm 1 with the pre-correction's
    D^{-1} replaced by an operator M1 and the post-correction's by M2 (= M_D^2
    = M_D^3) equals the dense product of the three factors, at one level
    (p = 1, M_S = A_0^{-1}); with exact D^{-1} in both places it is the
    block inverse with S replaced by A_0."""
    import scipy.sparse as sp
    prob = S.make_problem(4, 2, 0.3, 0.5)
    A = so.kl_matrices(prob.rowptr, prob.colidx, prob.vals)
    G = chaos.g_matrices(2, 1)
    _, off = chaos.multi_indices(2, 1)
    n, P = prob.n, G[0].shape[0]
    K = so.global_matrix_chaos_major(A, G).toarray()
    e = n * off[1]
    A0, B, C, D = K[:e, :e], K[:e, e:], K[e:, :e], K[e:, e:]
    rng = np.random.default_rng(4)
    X = rng.standard_normal((D.shape[0], D.shape[0]))
    M1 = np.linalg.inv(D) + 1e-2 * (X + X.T)         # two different symmetric approximations of D^{-1}
    M2 = np.diag(1.0 / np.diag(D))
    blk = lambda Md: (lambda l, Y: (Md @ Y.T.ravel()).reshape(Y.shape[1], n).T)
    R = S.random_block(n, P, seed=2)
    U = hsc.hsc_apply(A, G, off, R, dsolve_pre=blk(M1), dsolve_post=blk(M2))
    Md = hsc.general_prec(A0, B, C, np.linalg.inv(A0), M1, M2, M2)
    ref = (Md @ R.T.ravel()).reshape(P, n).T
    assert np.abs(U - ref).max() <= 1e-12 * np.abs(ref).max()
    Dinv = np.linalg.inv(D)
    exact = hsc.general_prec(A0, B, C, np.linalg.inv(A0), Dinv, Dinv, Dinv)
    assert np.abs(exact - hsc.block_inverse(A0, B, C, D, S_inv=np.linalg.inv(A0))).max() <= 1e-12 * np.abs(exact).max()


@pytest.mark.parametrize("M,p", [(2, 2), (2, 3), (3, 2)])
def test_algorithm1_gpc_equals_recursive_block_inverse(M, p):
    """Sec. 6, lognormal case (Remark K-L): with the coefficient expanded to
    degree 2p in Hermite chaos the global matrix is block dense, B_l and C_l
    couple degree l with every lower degree and D_l couples the chaos
    polynomials of one degree. Algorithm 1 with the assembled D_l solves equals
    the dense recursion of eq. (block-inverse) with S_{l-1} -> A_{l-1}, and
    M_bGS equals its closed form (D + U)^{-1} D (D + L)^{-1}."""
    prob = S.make_lognormal_problem(4, M, 0.5, 0.5, 2 * p)
    A = so.kl_matrices(prob.rowptr, prob.colidx, prob.vals)
    G = chaos.gpc_g_matrices(M, p, 2 * p)
    _, off = chaos.multi_indices(M, p)
    n, P = prob.n, G[0].shape[0]
    # the general case: D_p is not block diagonal and B_p reaches degree p - 2
    Dp = [g[off[p]:off[p + 1], off[p]:off[p + 1]].toarray() for g in G]
    assert any(np.abs(d - np.diag(np.diag(d))).max() > 0 for d in Dp)
    assert any(g[off[p - 2]:off[p - 1], off[p]:off[p + 1]].nnz for g in G)
    K = so.global_matrix_chaos_major(A, G).toarray()
    R = S.random_block(n, P, seed=31)
    Z = hsc.hsc_apply(A, G, off, R, general=True)
    Md = hsc.hsc_dense_recursive(K, n, off)
    z = (Md @ R.T.ravel()).reshape(P, n).T
    assert np.abs(Z - z).max() <= 1e-11 * np.abs(z).max()
    Mb = hsc.bgs_dense(K, n, P)
    ref = (Mb @ R.T.ravel()).reshape(P, n).T
    assert np.abs(hsc.bgs_apply(A, G, R) - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("M,p", [(2, 2), (3, 2)])
def test_schur_reduced_iteration_is_preconditioned_by_algorithm1(M, p):
    """Sec. 5, eq. (global-Schur-system): the reduced iteration on S_{p-1} is
    preconditioned by Algorithm 1 on the levels 0..p-1; run to full accuracy
    on a tiny system its Lanczos estimate is the condition number of
    M_{p-1} S_{p-1} formed densely (eq. (block-inverse) recursion for M_{p-1},
    S_{p-1} = A_{p-1} - B_p D_p^{-1} C_p from the assembled matrix). The Ritz
    values lie inside the spectrum, so the estimate is at most that number
    and, after the few iterations a tiny system needs, within 1 % below it;
    the mean-based preconditioner would give about twice the value."""
    prob = S.make_problem(4, M, 0.4, 0.5)
    A = so.kl_matrices(prob.rowptr, prob.colidx, prob.vals)
    G = chaos.g_matrices(M, p)
    _, off = chaos.multi_indices(M, p)
    n = prob.n
    F = S.random_block(n, G[0].shape[0], seed=12)
    _, info = hsc.schur_reduced_solve(A, G, off, F, tol=1e-14, maxit=200)
    K = so.global_matrix_chaos_major(A, G).toarray()
    e = n * off[p]
    Sd = K[:e, :e] - K[:e, e:] @ np.linalg.solve(K[e:, e:], K[e:, :e])
    Mr = hsc.hsc_dense_recursive(K[:e, :e], n, off[:p + 1])
    ev = np.sort(np.linalg.eigvals(Mr @ Sd).real)
    kappa = ev[-1] / ev[0]
    est = krylov.lanczos_kappa(info["alpha"], info["beta"])
    assert 0.99 * kappa <= est <= kappa * (1 + 1e-9)
    evm = np.sort(np.linalg.eigvals(np.kron(np.eye(off[p]), np.linalg.inv(A[0].toarray())) @ Sd).real)
    assert evm[-1] / evm[0] > 1.5 * kappa


@pytest.mark.parametrize("M", [1, 2, 3])
def test_schur_constants_are_the_spectrum_of_one_level(M):
    """Eq. (AS-ineq) at one level (p = 1): A_1 = L diag(S_0, D_1) L^T with
    M_1 = L^{-T} diag(A_0^{-1}, D_1^{-1}) L^{-1} gives spec(M_1 A_1) =
    spec(A_0^{-1} S_0) U {1}, the eigenvalue 1 once per degree-1 unknown; so
    the pencil constants (c_{0,1}, c_{0,2}) are the smallest and the largest
    eigenvalue of M_1 A_1 once the unit ones are set aside."""
    prob = S.make_problem(4, M, 0.5, 0.5)
    A = so.kl_matrices(prob.rowptr, prob.colidx, prob.vals)
    G = chaos.g_matrices(M, 1)
    _, off = chaos.multi_indices(M, 1)
    n = prob.n
    K = so.global_matrix_chaos_major(A, G).toarray()
    ev = np.sort(np.linalg.eigvals(hsc.hsc_dense_recursive(K, n, off) @ K).real)
    unit = np.abs(ev - 1.0) < 1e-9
    assert unit.sum() == n * M
    rest = ev[~unit]
    (c1, c2), = hsc.schur_constants(K, n, off)
    assert rest.size == n and c2 < 1 - 1e-6
    assert c1 == pytest.approx(rest[0], rel=1e-10) and c2 == pytest.approx(rest[-1], rel=1e-10)


def test_general_prec_factors_sit_where_the_paper_puts_them():
    """Eq. (general-prec) with three different approximations M_D^1, M_D^2,
    M_D^3 of D^{-1}: on [0; y] with C = 0 the product gives
    [-M_S B M_D^1 y; M_D^2 y] (M_D^1 in the pre-correction, M_D^2 in the middle
    factor), and on [x; 0] with B = 0 it gives [M_S x; -M_D^3 C M_S x] (M_D^3 in
    the post-correction)."""
    rng = np.random.default_rng(9)
    na, nd = 4, 3
    A0 = rng.standard_normal((na, na))
    B = rng.standard_normal((na, nd))
    C = rng.standard_normal((nd, na))
    MS = rng.standard_normal((na, na))
    M1, M2, M3 = (rng.standard_normal((nd, nd)) for _ in range(3))
    x, y = rng.standard_normal(na), rng.standard_normal(nd)
    P = hsc.general_prec(A0, B, np.zeros_like(C), MS, M1, M2, M3)
    assert np.allclose(P @ np.concatenate([np.zeros(na), y]), np.concatenate([-MS @ B @ M1 @ y, M2 @ y]),
                       rtol=0, atol=1e-13)
    P = hsc.general_prec(A0, np.zeros_like(B), C, MS, M1, M2, M3)
    assert np.allclose(P @ np.concatenate([x, np.zeros(nd)]), np.concatenate([MS @ x, -M3 @ C @ MS @ x]),
                       rtol=0, atol=1e-13)
