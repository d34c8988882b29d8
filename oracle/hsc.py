"""Hierarchical Schur complement preconditioner (oracle; test infrastructure only).

Algorithm 1 (Sec. 4) with exact solves of the diagonal blocks, the block
inverse of eq. (block-inverse) for the pins, and the Schur complements and the
spectral-equivalence constants of eq. (AS-ineq) that Theorem 1 uses.

Reading of Algorithm 1 used here and on the GPU (the paper writes it without
naming the storage): one working residual ``r`` holds ``r_P``; the
pre-correction at level ``l`` overwrites the degree ``< l`` part with
``g_{l-1} = r_l^{l-1} - B_l D_l^{-1} r_l^l``; in the post-correction loop,
``r_l^l`` is the degree-``l`` part of that working residual, i.e. of ``g_l``
for ``l < P`` and of the input for ``l = P``.
"""
from __future__ import annotations

from typing import Callable, List, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


class A0Solver:
    """Exact ``A_0^{-1}`` applied to the columns of an ``n x w`` block
    (sparse LU of the mean-value matrix; eq. (mean-value-problem))."""

    def __init__(self, A0: sp.spmatrix):
        self.lu = spla.splu(sp.csc_matrix(A0))

    def __call__(self, B: np.ndarray) -> np.ndarray:
        if B.shape[1] == 0:
            return B.copy()
        return self.lu.solve(np.ascontiguousarray(B))


def _offdiag_apply(A, G, rows, cols, X):
    """``sum_k A_k X G_k[rows, cols]^T``: the block of ``A_l`` with chaos rows
    ``rows`` and chaos columns ``cols`` applied to ``X`` (eq.
    (global-matrix-hierarchy), blocks ``B_l`` and ``C_l``)."""
    Y = np.zeros((A[0].shape[0], rows.stop - rows.start))
    for Ak, Gk in zip(A, G):
        sub = Gk[rows, cols]
        if sub.nnz:
            Y += (sub @ (Ak @ X).T).T
    return Y


def _diag_block_solver(A, G, lo: int, hi: int, general: bool, a0solve: A0Solver):
    """Exact ``D_l^{-1}``. With ``general`` the block
    ``D_l = sum_k A_k (x) G_k[lvl, lvl]`` is assembled and factored as it
    stands; otherwise the Lemma of Sec. 3 (``d_l`` diagonal, so
    ``D_l = I (x) A_0`` in the normalised basis) gives independent column
    solves with ``A_0``."""
    if not general:
        return a0solve
    n = A[0].shape[0]
    w = hi - lo
    D = None
    for Ak, Gk in zip(A, G):
        sub = Gk[lo:hi, lo:hi]
        if sub.nnz:
            t = sp.kron(Ak, sub, format="csc")
            D = t if D is None else D + t
    lu = spla.splu(sp.csc_matrix(D))
    return lambda X: lu.solve(np.ascontiguousarray(X).ravel()).reshape(n, w)


def hsc_apply(A, G, off, R: np.ndarray, general: bool = False,
              a0solve: Optional[A0Solver] = None,
              dsolve: Optional[Callable[[int, np.ndarray], np.ndarray]] = None,
              dsolve_pre: Optional[Callable[[int, np.ndarray], np.ndarray]] = None,
              dsolve_post: Optional[Callable[[int, np.ndarray], np.ndarray]] = None) -> np.ndarray:
    """Algorithm 1: ``M_P : r_P -> u_P``.

    ``off`` are the degree offsets of the chaos columns. ``dsolve(l, X)``
    replaces the exact ``D_l^{-1}`` (and ``A_0^{-1}`` for ``l = 0``) when given,
    which is how the inexact inner solves are modelled. ``dsolve_pre`` and
    ``dsolve_post`` replace it in the pre-correction (``M_D^1`` of eq.
    (general-prec), Sec. 5) and in the post-correction (``M_D^2 = M_D^3``,
    applied to ``r_l - C_l u``) only, for the variants of Sec. 5 that use, e.g.,
    the mean-value preconditioner ``M_0`` there.
    """
    n, P = R.shape
    p = len(off) - 2
    if a0solve is None and dsolve is None:
        a0solve = A0Solver(A[0])
    if dsolve is None:
        solvers = {l: _diag_block_solver(A, G, off[l], off[l + 1], general, a0solve) for l in range(1, p + 1)}
        solvers[0] = a0solve
        dsolve = lambda l, X: solvers[l](X)
    pre_solve = dsolve_pre or dsolve
    post_solve = dsolve_post or dsolve
    r = np.array(R, dtype=np.float64, copy=True)
    # first loop, l = P..1: pre-correction
    for l in range(p, 0, -1):
        lo, hi = off[l], off[l + 1]
        y = pre_solve(l, r[:, lo:hi])                                # D_l^{-1} r_l^l (M_D^1)
        r[:, :lo] -= _offdiag_apply(A, G, slice(0, lo), slice(lo, hi), y)   # g_{l-1}
    # mean-value problem A_0 u_0 = g_0
    u = np.zeros((n, P))
    u[:, 0:off[1]] = dsolve(0, r[:, 0:off[1]])
    # second loop, l = 1..P: post-correction
    for l in range(1, p + 1):
        lo, hi = off[l], off[l + 1]
        t = r[:, lo:hi] - _offdiag_apply(A, G, slice(lo, hi), slice(0, lo), u[:, :lo])
        u[:, lo:hi] = post_solve(l, t)                               # M_D^2 = M_D^3
    return u


def schur_reduced_solve(A, G, off, F: np.ndarray, tol: float = 1e-8, maxit: int = 500):
    """The a-priori reduction of Sec. 5, eq. (global-Schur-system): eliminate
    the degree-p unknowns ``u_P^P`` and iterate on
    ``S_{p-1} u_{p-1} = g_{p-1}`` with ``S_{p-1} = A_{p-1} - B_p D_p^{-1} C_p``
    and ``g_{p-1} = f^{p-1} - B_p D_p^{-1} f^p`` (exact ``D_p^{-1}``), by
    flexible CG preconditioned with Algorithm 1 on the levels ``1..p-1``;
    then recover ``u^p = D_p^{-1} (f^p - C_p u_{p-1})``. Returns the full
    ``n x P`` solution and the CG information of the reduced iteration."""
    from .krylov import fcg
    p = len(off) - 2
    if p < 1:
        raise ValueError("the reduction needs p >= 1")
    lo = off[p]
    a0 = A0Solver(A[0])
    dsolve = _diag_block_solver(A, G, off[p], off[p + 1], False, a0)
    sub_G = [g[:lo, :lo] for g in G]
    off_r = off[:p + 1]

    def S(V):
        y = sg_apply_sub(A, sub_G, V)
        y -= _offdiag_apply(A, G, slice(0, lo), slice(lo, off[p + 1]),
                            dsolve(_offdiag_apply(A, G, slice(lo, off[p + 1]), slice(0, lo), V)))
        return y

    g = F[:, :lo] - _offdiag_apply(A, G, slice(0, lo), slice(lo, off[p + 1]), dsolve(F[:, lo:]))
    u_r, info = fcg(S, g, lambda R: hsc_apply(A, sub_G, off_r, R, a0solve=a0), tol=tol, maxit=maxit)
    U = np.zeros_like(F)
    U[:, :lo] = u_r
    U[:, lo:] = dsolve(F[:, lo:] - _offdiag_apply(A, G, slice(lo, off[p + 1]), slice(0, lo), u_r))
    return U, info


def sg_apply_sub(A, G, U):
    """``sum_k A_k U G_k^T`` (the MAT-VEC of eq. (global-system)) for blocks
    ``G_k`` of any square size."""
    Y = np.zeros((A[0].shape[0], U.shape[1]))
    for Ak, Gk in zip(A, G):
        if Gk.nnz:
            Y += (Gk @ (Ak @ U).T).T
    return Y


def bgs_apply(A, G, R: np.ndarray, dsolve: Optional[Callable[[int, np.ndarray], np.ndarray]] = None) -> np.ndarray:
    """Block symmetric Gauss-Seidel with zero initial guess, ``M_bGS`` of
    Sec. 6 (the paper's main comparison preconditioner): the blocks are the
    ``P x P`` blocks ``K^(j,l) = sum_k c_kjl A_k`` of eq. (global-matrix), one
    per pair of chaos indices, swept in the chaos order, forward
    ``j = 0..P-1`` and then backward ``j = P-1..0``:

        forward   u_j = K_jj^{-1} (r_j - sum_{l<j} K_jl u_l)
        backward  u_j = K_jj^{-1} (r_j - sum_{l<j} K_jl u_l - sum_{l>j} K_jl u_l)

    where the backward sweep reads the forward values for ``l < j`` and its
    own new values for ``l > j``. ``dsolve(j, x)`` replaces the exact
    ``K_jj^{-1}`` (inexact inner solves)."""
    n, P = R.shape
    Gd = [g.toarray() for g in G]

    def block(j, l):
        out = None
        for Ak, Gk in zip(A, Gd):
            c = Gk[j, l]
            if c != 0.0:
                out = c * Ak if out is None else out + c * Ak
        return out

    if dsolve is None:
        lus = {}

        def dsolve(j, x):
            key = tuple(Gk[j, j] for Gk in Gd)
            if key not in lus:
                lus[key] = spla.splu(sp.csc_matrix(block(j, j)))
            return lus[key].solve(np.ascontiguousarray(x))

    coupled = [[l for l in range(P) if l != j and any(Gk[j, l] != 0.0 for Gk in Gd)] for j in range(P)]
    u = np.zeros((n, P))
    for j in range(P):
        t = R[:, j].copy()
        for l in coupled[j]:
            if l < j:
                t -= block(j, l) @ u[:, l]
        u[:, j] = np.asarray(dsolve(j, t)).reshape(n)
    fwd = u.copy()
    for j in range(P - 1, -1, -1):
        t = R[:, j].copy()
        for l in coupled[j]:
            t -= block(j, l) @ (fwd[:, l] if l < j else u[:, l])
        u[:, j] = np.asarray(dsolve(j, t)).reshape(n)
    return u


def bgs_dense(K: np.ndarray, n: int, P: int) -> np.ndarray:
    """``M_bGS`` as a dense matrix (chaos-major ``K``): symmetric Gauss-Seidel
    with zero initial guess is ``(D + U)^{-1} D (D + L)^{-1}`` for the block
    diagonal ``D`` and the strictly lower / upper block parts ``L``, ``U``."""
    D = np.zeros_like(K)
    Lo = np.zeros_like(K)
    for j in range(P):
        for l in range(P):
            blk = K[j * n:(j + 1) * n, l * n:(l + 1) * n]
            if j == l:
                D[j * n:(j + 1) * n, l * n:(l + 1) * n] = blk
            elif l < j:
                Lo[j * n:(j + 1) * n, l * n:(l + 1) * n] = blk
    Up = K - D - Lo
    return np.linalg.solve(D + Up, D @ np.linalg.inv(D + Lo))


def mean_apply(A, R: np.ndarray, a0solve: Optional[A0Solver] = None) -> np.ndarray:
    """Mean-based preconditioner ``M_m = I (x) A_0^{-1}`` (Sec. 6): one exact
    mean-value solve per chaos column."""
    if a0solve is None:
        a0solve = A0Solver(A[0])
    return a0solve(R)


# ---------------------------------------------------------------------------
# Dense forms for the pins (tiny problems only), chaos-major as in the paper
# ---------------------------------------------------------------------------

def block_inverse(A: np.ndarray, B: np.ndarray, C: np.ndarray, D: np.ndarray,
                  S_inv: Optional[np.ndarray] = None) -> np.ndarray:
    """Eq. (block-inverse): the product of the post-correction, correction and
    pre-correction factors. With ``S_inv = (A - B D^{-1} C)^{-1}`` it is the
    exact inverse of ``[[A, B], [C, D]]``; any other ``S_inv`` gives the
    approximation used by Algorithm 1."""
    Dinv = np.linalg.inv(D)
    if S_inv is None:
        S_inv = np.linalg.inv(A - B @ Dinv @ C)
    na, nd = A.shape[0], D.shape[0]
    post = np.block([[np.eye(na), np.zeros((na, nd))], [-Dinv @ C, np.eye(nd)]])
    mid = np.block([[S_inv, np.zeros((na, nd))], [np.zeros((nd, na)), Dinv]])
    pre = np.block([[np.eye(na), -B @ Dinv], [np.zeros((nd, na)), np.eye(nd)]])
    return post @ mid @ pre


def general_prec(A: np.ndarray, B: np.ndarray, C: np.ndarray, MS: np.ndarray, MD1: np.ndarray,
                 MD2: np.ndarray, MD3: np.ndarray) -> np.ndarray:
    """Eq. (general-prec) of Sec. 5 as a dense matrix: the post-correction
    factor with ``M_D^3``, the middle factor ``diag(M_S, M_D^2)`` and the
    pre-correction factor with ``M_D^1`` (``A`` only fixes the size of the
    first block)."""
    na, nd = A.shape[0], MD2.shape[0]
    post = np.block([[np.eye(na), np.zeros((na, nd))], [-MD3 @ C, np.eye(nd)]])
    mid = np.block([[MS, np.zeros((na, nd))], [np.zeros((nd, na)), MD2]])
    pre = np.block([[np.eye(na), -B @ MD1], [np.zeros((nd, na)), np.eye(nd)]])
    return post @ mid @ pre


def hsc_dense_recursive(K: np.ndarray, n: int, off) -> np.ndarray:
    """``M_P`` as a dense matrix by the recursion of Sec. 4: eq.
    (block-inverse) at every level with ``S_{l-1}^{-1}`` replaced by the
    preconditioner of ``A_{l-1}``, down to ``A_0^{-1}``. ``K`` is the
    chaos-major global matrix."""
    def M(l):
        e = n * off[l + 1]
        if l == 0:
            return np.linalg.inv(K[:e, :e])
        s = n * off[l]
        return block_inverse(K[:s, :s], K[:s, s:e], K[s:e, :s], K[s:e, s:e], S_inv=M(l - 1))
    return M(len(off) - 2)


def schur_constants(K: np.ndarray, n: int, off) -> List[tuple]:
    """``(c_{l,1}, c_{l,2})`` of eq. (AS-ineq) for ``l = 0..P-1``: the extreme
    eigenvalues of the pencil ``S_l v = mu A_l v`` with
    ``S_l = A_l - B_{l+1} D_{l+1}^{-1} C_{l+1}``."""
    out = []
    p = len(off) - 2
    for l in range(p):
        s, e = n * off[l + 1], n * off[l + 2]
        A_l = K[:s, :s]
        B = K[:s, s:e]
        C = K[s:e, :s]
        D = K[s:e, s:e]
        S = A_l - B @ np.linalg.solve(D, C)
        mu = sla.eigh(0.5 * (S + S.T), 0.5 * (A_l + A_l.T), eigvals_only=True)
        out.append((float(mu[0]), float(mu[-1])))
    return out
