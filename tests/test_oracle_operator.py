"""Pins of the oracle's SG operator against the paper's explicit block matrix,
symmetry and definiteness, and the direct solve."""
import numpy as np
import pytest
import scipy.sparse as sp

import sg_inputs as S
from oracle import chaos, sg_operator as so


def _small(ne=4, M=2, p=3, sigma=0.3, corr=0.5):
    prob = S.make_problem(ne, M, sigma, corr)
    A = so.kl_matrices(prob.rowptr, prob.colidx, prob.vals)
    G = chaos.g_matrices(M, p)
    _, off = chaos.multi_indices(M, p)
    return prob, A, G, off


@pytest.mark.parametrize("ne,M,p", [(4, 2, 3), (8, 3, 2), (4, 1, 4)])
def test_sg_apply_matches_block_matrix_of_the_paper(ne, M, p):
    """eq. (global-matrix) with blocks K^(j,l) = sum_i c_ijl K_i, chaos-major,
    against the MAT-VEC form used everywhere else."""
    prob, A, G, off = _small(ne, M, p)
    n, P = prob.n, G[0].shape[0]
    U = S.random_block(n, P, seed=11)
    K = so.global_matrix_chaos_major(A, G)
    y_chaos = K @ U.T.ravel()                  # chaos-major vec: column l stacked
    Y = so.sg_apply(A, G, U)
    assert np.allclose(Y, y_chaos.reshape(P, n).T, rtol=0, atol=1e-13 * np.abs(Y).max())
    # space-major Kronecker form with the permutation between layouts
    Ks = so.global_matrix_space_major(A, G)
    perm = so.chaos_major_to_space_major(n, P)
    assert abs(Ks - K[perm][:, perm]).max() < 1e-15
    # K^(0,0) = K_0 (Sec. 2): the first diagonal block is the mean problem
    assert abs(K[:n, :n] - A[0]).max() == 0


def test_global_matrix_symmetric_positive_definite_cfg1_small():
    prob, A, G, off = _small(8, 3, 3, sigma=0.2, corr=0.5)
    K = so.global_matrix_space_major(A, G).toarray()
    assert np.abs(K - K.T).max() < 1e-15
    ev = np.linalg.eigvalsh(K)
    assert ev[0] > 0


def test_direct_solve_residual_and_linearity():
    prob, A, G, off = _small(8, 2, 3)
    F = S.make_rhs(prob, 3)
    U = so.direct_solve(A, G, F)
    R = F - so.sg_apply(A, G, U)
    assert np.linalg.norm(R) / np.linalg.norm(F) < 1e-13
    # the mean of the solution solves nothing simpler, but its degree-1 part is
    # driven only by the coupling: it must be nonzero when sigma > 0
    assert np.abs(U[:, off[1]:off[2]]).max() > 0


def test_level_blocks_sum_to_operator_without_diagonal():
    prob, A, G, off = _small(4, 3, 3)
    n, P = prob.n, G[0].shape[0]
    U = S.random_block(n, P, seed=5)
    Y = so.sg_apply(A, G, U)
    Y2 = A[0] @ U                               # G_0 = I: diagonal blocks
    p = len(off) - 2
    for lo in range(p + 1):
        for li in range(p + 1):
            if abs(lo - li) == 1:
                Y2[:, off[lo]:off[lo + 1]] += so.level_apply(A, G, off, lo, li, U[:, off[li]:off[li + 1]])
    assert np.allclose(Y, Y2, atol=1e-13)


def test_row_sampled_products_match_the_explicit_global_matrix():
    """The row-restricted products (used to check single rows of the
    full-size GPU products) against rows of the assembled Kronecker matrix
    sum_k A_k (x) G_k and of its level blocks (eq. (global-matrix-hierarchy))."""
    prob, A, G, off = _small(8, 3, 3)
    n, P = prob.n, G[0].shape[0]
    U = S.random_block(n, P, seed=21)
    rows = np.array([0, 5, 17, n - 1, 17])
    Ks = so.global_matrix_space_major(A, G)
    y = (Ks @ U.ravel()).reshape(n, P)
    Yr = so.sg_apply_rows(A, G, U, rows)
    assert np.allclose(Yr, y[rows], rtol=0, atol=1e-13 * np.abs(y).max())
    K = so.global_matrix_chaos_major(A, G).toarray()
    p = len(off) - 2
    for lo, li in [(p - 1, p), (p, p - 1), (0, 1)]:
        X = S.random_block(n, off[li + 1] - off[li], seed=lo + 7 * li)
        blk = K[off[lo] * n:off[lo + 1] * n, off[li] * n:off[li + 1] * n]
        y = (blk @ X.T.ravel()).reshape(off[lo + 1] - off[lo], n).T
        assert np.allclose(so.level_apply(A, G, off, lo, li, X, rows=rows), y[rows], rtol=0,
                           atol=1e-13 * np.abs(y).max())


def test_kl_matrices_hold_each_term_column():
    """Brute force over the stored nonzeros: (A_k)_{r, c_e} is vals[e, k] for
    every term k, and nothing else is stored."""
    prob = S.make_problem(4, 3, 0.3, 0.5)
    A = so.kl_matrices(prob.rowptr, prob.colidx, prob.vals)
    assert len(A) == 4
    for k, Ak in enumerate(A):
        D = Ak.toarray()
        seen = np.zeros_like(D, dtype=bool)
        for r in range(prob.n):
            for e in range(prob.rowptr[r], prob.rowptr[r + 1]):
                assert D[r, prob.colidx[e]] == prob.vals[e, k]
                seen[r, prob.colidx[e]] = True
        assert not np.any(D[~seen])
