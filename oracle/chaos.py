"""Polynomial chaos basis and triple products (oracle; test infrastructure only).

Sec. 2, eq. (gPC-u): the chaos basis is the set of tensor-product polynomials
of total degree at most ``p`` in ``M`` variables; their number is
``(M+p)! / (M! p!)``. Eq. (global-system): the SG matrix couples the spatial
matrices through ``c_ijk = E[psi_i psi_j psi_k]``; for the linear KL
expansion only ``psi_0 = 1`` and ``psi_{e_k} = xi_k`` appear as the first
index, so the operator is ``sum_k G_k (x) A_k`` with
``(G_k)_{jl} = E[xi_k psi_j psi_l]`` and ``G_0 = I``.

Ordering (the paper is silent inside one degree; this is the reading used on
both sides of the boundary): degrees ascending (graded, as Sec. 3 needs), and
inside one degree descending lexicographic order of ``(alpha_1..alpha_M)``, so
degree 1 is ``e_1, e_2, ..., e_M``.
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np
import scipy.sparse as sp

LEGENDRE = "legendre"
HERMITE = "hermite"


def _compositions_desc(d: int, M: int):
    """All alpha in N^M with |alpha| = d, descending lexicographic order."""
    if M == 1:
        yield (d,)
        return
    for a in range(d, -1, -1):
        for rest in _compositions_desc(d - a, M - 1):
            yield (a,) + rest


def multi_indices(M: int, p: int) -> Tuple[np.ndarray, np.ndarray]:
    """Graded multi-index table and level offsets.

    Returns ``alpha`` of shape ``(P, M)`` and ``off`` of length ``p + 2`` with
    the degree-``l`` block in rows ``off[l]:off[l+1]`` (Sec. 3, the splitting
    ``c_l = [[c_{l-1}, b_l^T], [b_l, d_l]]`` requires lower degrees first).
    """
    rows, off = [], [0]
    for d in range(p + 1):
        rows.extend(_compositions_desc(d, M) if M > 0 else ([()] if d == 0 else []))
        off.append(len(rows))
    alpha = np.array(rows, dtype=np.int64).reshape(len(rows), M)
    return alpha, np.array(off, dtype=np.int64)


def chaos_count(M: int, p: int) -> int:
    """Eq. (gPC-u): number of chaos polynomials ``(M+p)!/(M! p!)``."""
    return math.comb(M + p, M)


def xi_triple_1d(m: int, family: str) -> float:
    """``E[xi psi_m psi_{m+1}]`` for the normalised 1-D family.

    Legendre, ``xi ~ U(-sqrt3, sqrt3)``: ``psi_m(xi) = sqrt(2m+1) L_m(xi/sqrt3)``
    and ``t L_m = ((m+1) L_{m+1} + m L_{m-1}) / (2m+1)`` give
    ``sqrt3 (m+1) / sqrt((2m+1)(2m+3))``. Hermite, ``xi ~ N(0,1)``:
    ``psi_m = He_m / sqrt(m!)`` gives ``sqrt(m+1)``.
    """
    if family == LEGENDRE:
        return math.sqrt(3.0) * (m + 1) / math.sqrt((2 * m + 1) * (2 * m + 3))
    if family == HERMITE:
        return math.sqrt(m + 1.0)
    raise ValueError(family)


def g_matrices(M: int, p: int, family: str = LEGENDRE) -> List[sp.csr_matrix]:
    """``[G_0, G_1, ..., G_M]`` with ``(G_k)_{jl} = E[xi_k psi_j psi_l]``.

    By orthogonality in every coordinate other than ``k`` the entry is nonzero
    only if ``alpha_j`` and ``alpha_l`` differ in coordinate ``k`` alone and by
    one; its value is then the 1-D triple product at ``m = min``.
    """
    alpha, _ = multi_indices(M, p)
    P = alpha.shape[0]
    index = {tuple(a): i for i, a in enumerate(alpha)}
    Gs = [sp.identity(P, format="csr", dtype=np.float64)]
    for k in range(M):
        rows, cols, vals = [], [], []
        for j in range(P):
            a = alpha[j]
            for step in (+1, -1):
                b = a.copy()
                b[k] += step
                if b[k] < 0:
                    continue
                l = index.get(tuple(b))
                if l is None:
                    continue
                rows.append(j)
                cols.append(l)
                vals.append(xi_triple_1d(min(a[k], b[k]), family))
        Gs.append(sp.csr_matrix((vals, (rows, cols)), shape=(P, P)))
    return Gs


def block_counts(M: int, p: int, family: str = LEGENDRE) -> dict:
    """Block counts of the SG matrix (Sec. 6, Table 5 and Fig. 1).

    ``n_b``: nonzero blocks of ``c_P`` (entries ``sum_i c_ijk``);
    ``n_db``: diagonal blocks; ``n_m = n_b - n_db``: block matrix-vector
    products per HSC application; ``n_ds = 2 (n_db - 1) + 1``: block diagonal
    solves per HSC application (the two loops of Algorithm 1 plus the mean
    solve).
    """
    Gs = g_matrices(M, p, family)
    pattern = sum(abs(G) for G in Gs)
    pattern.eliminate_zeros()
    n_b = int(pattern.nnz)
    n_db = int(Gs[0].shape[0])
    return dict(n_b=n_b, n_db=n_db, n_m=n_b - n_db, n_ds=2 * (n_db - 1) + 1)


# ---------------------------------------------------------------------------
# General gPC coefficient expansions (Remark K-L, Sec. 6 lognormal case)
# ---------------------------------------------------------------------------

def hermite_triple_1d(a: int, b: int, c: int) -> float:
    """``E[psi_a psi_b psi_c]`` for the normalised Hermite polynomials
    ``psi_m = He_m / sqrt(m!)`` of ``xi ~ N(0,1)``: with ``s = (a+b+c)/2`` it is
    ``sqrt(a! b! c!) / ((s-a)! (s-b)! (s-c)!)`` when ``s`` is an integer not
    below any of ``a, b, c``, and zero otherwise (the classical product formula
    of Hermite polynomials)."""
    t = a + b + c
    if t % 2:
        return 0.0
    s2 = t // 2
    if s2 < a or s2 < b or s2 < c:
        return 0.0
    return math.sqrt(math.factorial(a) * math.factorial(b) * math.factorial(c)) / (
        math.factorial(s2 - a) * math.factorial(s2 - b) * math.factorial(s2 - c))


def gpc_g_matrices(M: int, p: int, q: int) -> List[sp.csr_matrix]:
    """``[G_i]`` for the coefficient basis of total degree ``<= q`` (graded
    order, as the solution basis) with ``(G_i)_{jl} = E[psi_i psi_j psi_l]``
    over the solution basis of degree ``<= p``, normalised Hermite chaos:
    the SG matrix of eq. (global-system) for a gPC-expanded coefficient
    ``k = sum_i k_i psi_i`` (Remark K-L). The triple product of tensor-product
    polynomials is the product of the 1-D ones over the coordinates."""
    alpha, _ = multi_indices(M, p)
    gamma, _ = multi_indices(M, q)
    P = alpha.shape[0]
    out = []
    for g in gamma:
        rows, cols, vals = [], [], []
        for j in range(P):
            for l in range(P):
                v = 1.0
                for k in range(M):
                    v *= hermite_triple_1d(int(g[k]), int(alpha[j][k]), int(alpha[l][k]))
                    if v == 0.0:
                        break
                if v != 0.0:
                    rows.append(j)
                    cols.append(l)
                    vals.append(v)
        out.append(sp.csr_matrix((vals, (rows, cols)), shape=(P, P)))
    return out
