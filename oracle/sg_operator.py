"""The SG operator, the explicit global matrix and the direct solve (oracle).

Test infrastructure only. Layout: a coefficient block ``U`` is ``n x P``,
row-major, spatial index slow and chaos index fast. In this layout the global
system of eq. (global-system) reads ``Y = sum_k A_k U G_k^T``, because
``Y(:, l) = sum_k sum_j c_{kjl} A_k U(:, j)`` and ``G_k`` is symmetric.
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def kl_matrices(rowptr, colidx, vals) -> List[sp.csr_matrix]:
    """``[A_0..A_M]`` as scipy CSR from the shared pattern and ``vals[nnz][M+1]``."""
    n = len(rowptr) - 1
    return [sp.csr_matrix((np.ascontiguousarray(vals[:, k]), colidx, rowptr), shape=(n, n))
            for k in range(vals.shape[1])]


def sg_apply(A: Sequence[sp.spmatrix], G: Sequence[sp.spmatrix], U: np.ndarray) -> np.ndarray:
    """MAT-VEC of the SG system (eq. (global-system) with the remark after
    eq. (global-matrix-block)): ``Y = sum_k A_k U G_k^T``; neither the global
    matrix nor any block ``K^(j,k)`` is formed."""
    Y = np.zeros((A[0].shape[0], U.shape[1]))
    for Ak, Gk in zip(A, G):
        Y += (Gk @ (Ak @ U).T).T
    return Y


def sg_apply_rows(A: Sequence[sp.spmatrix], G: Sequence[sp.spmatrix], U: np.ndarray, rows) -> np.ndarray:
    """Rows ``rows`` of the MAT-VEC of eq. (global-system):
    ``Y[rows] = sum_k A_k[rows, :] U G_k^T``. Row ``r`` of the product needs
    only row ``r`` of every ``A_k``, so a sample of rows (or a block of
    them) is computed without the rest."""
    rows = np.asarray(rows)
    Y = np.zeros((len(rows), U.shape[1]))
    for Ak, Gk in zip(A, G):
        Y += (Gk @ (Ak[rows] @ U).T).T
    return Y


def global_matrix_chaos_major(A: Sequence[sp.spmatrix], G: Sequence[sp.spmatrix]) -> sp.csr_matrix:
    """Eq. (global-matrix): the block matrix with blocks
    ``K^(j,l) = sum_i c_ijl K_i`` (eq. (global-matrix-block)), unknowns
    ordered chaos-major ``[u_0; u_1; ...; u_P-1]`` as in the paper."""
    P = G[0].shape[0]
    Gd = [g.toarray() for g in G]
    blocks = [[None] * P for _ in range(P)]
    for j in range(P):
        for l in range(P):
            blk = None
            for Ak, Gk in zip(A, Gd):
                c = Gk[j, l]
                if c != 0.0:
                    blk = c * Ak if blk is None else blk + c * Ak
            blocks[j][l] = blk
    n = A[0].shape[0]
    for j in range(P):
        if blocks[j][j] is None:
            blocks[j][j] = sp.csr_matrix((n, n))
    return sp.bmat(blocks, format="csr")


def chaos_major_to_space_major(n: int, P: int) -> np.ndarray:
    """Permutation ``perm`` with ``x_space[i] = x_chaos[perm[i]]`` where
    space-major index is ``r*P + l`` and chaos-major index is ``l*n + r``."""
    r, l = np.meshgrid(np.arange(n), np.arange(P), indexing="ij")
    return (l * n + r).ravel()


def global_matrix_space_major(A, G) -> sp.csr_matrix:
    """The global matrix in this build's layout, ``sum_k A_k (x) G_k``."""
    out = None
    for Ak, Gk in zip(A, G):
        t = sp.kron(Ak, Gk, format="csr")
        out = t if out is None else out + t
    return out.tocsr()


def direct_solve(A, G, F: np.ndarray) -> np.ndarray:
    """The exact solution of ``sum_k A_k U G_k^T = F`` by a sparse direct solve
    of the assembled global matrix (the definition of the result)."""
    n, P = F.shape
    K = global_matrix_space_major(A, G).tocsc()
    x = spla.spsolve(K, F.ravel())
    return x.reshape(n, P)


def level_apply(A, G, off, lvl_out: int, lvl_in: int, X: np.ndarray, rows=None) -> np.ndarray:
    """Off-diagonal block product between degree levels (Sec. 3,
    eq. (global-matrix-hierarchy)): output rows are the degree-``lvl_out``
    chaos columns, inputs the degree-``lvl_in`` ones; returns
    ``sum_k A_k X G_k[out, in]^T`` of shape ``n x w_out`` (only the spatial
    rows ``rows`` when given, from the same rows of the ``A_k``)."""
    o0, o1 = off[lvl_out], off[lvl_out + 1]
    i0, i1 = off[lvl_in], off[lvl_in + 1]
    nr = A[0].shape[0] if rows is None else len(rows)
    Y = np.zeros((nr, o1 - o0))
    for Ak, Gk in zip(A, G):
        sub = Gk[o0:o1, i0:i1]
        if sub.nnz:
            Ar = Ak if rows is None else Ak[np.asarray(rows)]
            Y += (sub @ (Ar @ X).T).T
    return Y
