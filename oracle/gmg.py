"""Geometric multigrid V-cycle for the mean-value matrix ``A_0`` (oracle;
test infrastructure only).

The paper leaves the mean-value preconditioner ``M_0`` open (Sec. 5: "we do
not advocate any specific choice"; Sec. 6 used none, diagonal and exact LU).
The reading used by this build for the inner solves is one symmetric V-cycle:

* grids: the ``ne x ne`` Q1 grid and its coarsenings ``ne/2, ne/4, ..., 2``
  (``ne`` a power of two), interior nodes lexicographic with ``x`` fastest;
* prolongation ``P``: bilinear interpolation from the coarse interior nodes
  (fine nodes ``(2I, 2J)``) with zero Dirichlet values on the boundary;
  restriction ``R = P^T``;
* coarse operators: Galerkin products ``A_{g+1} = P^T A_g P``;
* smoother: ``nu`` sweeps of weighted Jacobi ``x += omega D^{-1} (b - A x)``
  before and after the coarse correction (so the cycle is symmetric);
* coarsest grid (one interior node for a square grid): exact solve.
"""
from __future__ import annotations

from typing import List

import numpy as np
import scipy.sparse as sp


def _w1d(i: int, I: int) -> float:
    d = abs(i - 2 * I)
    return 1.0 if d == 0 else (0.5 if d == 1 else 0.0)


def prolongation(ne: int) -> sp.csr_matrix:
    """Bilinear prolongation from the ``ne/2`` grid to the ``ne`` grid, both
    interior-only: ``P[(i,j),(I,J)] = w(i,I) w(j,J)`` with ``w = 1`` at
    ``i = 2I`` and ``1/2`` at ``|i - 2I| = 1``."""
    m, mc = ne - 1, ne // 2 - 1
    rows, cols, vals = [], [], []
    for J in range(1, mc + 1):
        for I in range(1, mc + 1):
            c = (J - 1) * mc + (I - 1)
            for j in range(2 * J - 1, 2 * J + 2):
                for i in range(2 * I - 1, 2 * I + 2):
                    rows.append((j - 1) * m + (i - 1))
                    cols.append(c)
                    vals.append(_w1d(i, I) * _w1d(j, J))
    return sp.csr_matrix((vals, (rows, cols)), shape=(m * m, mc * mc))


class Level:
    def __init__(self, A: sp.csr_matrix, ne: int, P: sp.csr_matrix = None):
        self.A = sp.csr_matrix(A)
        self.ne = ne
        self.P = P                      # prolongation from the next coarser level into this one
        self.dinv = 1.0 / self.A.diagonal()


def hierarchy(A0: sp.spmatrix, ne: int) -> List[Level]:
    """Galerkin hierarchy ``A_{g+1} = P_g^T A_g P_g`` down to ``ne = 2``."""
    if ne < 2 or (ne & (ne - 1)) != 0:
        raise ValueError("ne must be a power of two >= 2")
    levels = [Level(A0, ne)]
    while levels[-1].ne > 2:
        fine = levels[-1]
        P = prolongation(fine.ne)
        fine.P = P
        Ac = (P.T @ fine.A @ P).tocsr()
        levels.append(Level(Ac, fine.ne // 2))
    return levels


def vcycle(levels: List[Level], b: np.ndarray, nu: int = 2, omega: float = 0.8, g: int = 0) -> np.ndarray:
    """One V-cycle with zero initial guess on level ``g`` applied to ``b``
    (a vector or an ``n x w`` block, columns independent)."""
    L = levels[g]
    if g == len(levels) - 1:
        return np.linalg.solve(L.A.toarray(), b)
    dinv = L.dinv if b.ndim == 1 else L.dinv[:, None]
    x = np.zeros_like(b, dtype=np.float64)
    for _ in range(nu):
        x = x + omega * dinv * (b - L.A @ x)
    r = b - L.A @ x
    xc = vcycle(levels, L.P.T @ r, nu, omega, g + 1)
    x = x + L.P @ xc
    for _ in range(nu):
        x = x + omega * dinv * (b - L.A @ x)
    return x
