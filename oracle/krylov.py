"""Outer flexible CG, the Lanczos condition estimate and the inner batched PCG
(oracle; test infrastructure only).

Sec. 5: the HSC preconditioner with inner Krylov loops changes from one
application to the next, so the outer method is flexible CG (Notay); the
paper reports that standard CG behaved the same. Sec. 6: iterations stop at
relative residual ``1e-8`` and the condition number is estimated from the
Lanczos sequence of CG.

Readings (the paper is silent): the residual norm is the 2-norm of the
recursively updated residual; the flexible ``beta`` is the Polak-Ribiere form
``z_{k+1}^T (r_{k+1} - r_k) / (z_k^T r_k)``; the iteration count is the number
of operator applications.
"""
from __future__ import annotations

from typing import Callable, Optional

import numpy as np


def fcg(apply_A: Callable, f: np.ndarray, apply_M: Optional[Callable] = None, tol: float = 1e-8,
        maxit: int = 1000, flexible: bool = True, x0: Optional[np.ndarray] = None):
    """Preconditioned (flexible) CG on ``A x = f`` for SPD ``A``.

    Returns ``(x, info)`` with ``info['iters']``, the relative residual
    history ``info['res']`` (entry 0 is the initial one), and the CG
    coefficients ``info['alpha']``, ``info['beta']`` for the Lanczos
    estimate.
    """
    M = apply_M if apply_M is not None else (lambda r: r.copy())
    x = np.zeros_like(f) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    r = f - apply_A(x) if x0 is not None else np.array(f, dtype=np.float64, copy=True)
    fn = np.linalg.norm(f)
    res = [np.linalg.norm(r) / fn if fn > 0 else 0.0]
    alphas, betas = [], []
    info = dict(iters=0, res=res, alpha=alphas, beta=betas, converged=res[0] <= tol)
    if info["converged"]:
        return x, info
    z = M(r)
    p = z.copy()
    rho = float(np.vdot(z, r))
    for k in range(maxit):
        q = apply_A(p)
        pq = float(np.vdot(p, q))
        if not pq > 0:
            info["breakdown"] = True
            break
        alpha = rho / pq
        alphas.append(alpha)
        x += alpha * p
        r_old = r
        r = r - alpha * q
        res.append(np.linalg.norm(r) / fn)
        info["iters"] = k + 1
        if res[-1] <= tol:
            info["converged"] = True
            break
        z = M(r)
        rho_new = float(np.vdot(z, r))
        beta = (float(np.vdot(z, r - r_old)) if flexible else rho_new) / rho
        betas.append(beta)
        rho = rho_new
        p = z + beta * p
    return x, info


def lanczos_kappa(alphas, betas) -> float:
    """Condition estimate from the CG coefficients (Sec. 6): the Lanczos
    tridiagonal ``T`` has ``T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1}`` and
    ``T_{j,j+1} = sqrt(beta_j)/alpha_j``; return ``max eig / min eig``."""
    m = len(alphas)
    if m == 0:
        return 1.0
    T = np.zeros((m, m))
    for j in range(m):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < m:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(max(betas[j], 0.0)) / alphas[j]
    ev = np.linalg.eigvalsh(T)
    return float(ev[-1] / ev[0])


def pcg_columns(apply_A0: Callable, B: np.ndarray, apply_M0: Callable, tol: float,
                maxit: int, fixed_iters: int = 0):
    """Inner solves of the diagonal blocks (Sec. 5: independent preconditioned
    Krylov loops, one per diagonal block of ``D_l``), one column at a time.

    Conventions (the paper is silent; the GPU follows the same ones): zero
    initial guess; a column with ``||b|| = 0`` is done at entry with ``x = 0``;
    a column stops once ``||r|| <= tol ||b||``; with ``fixed_iters > 0`` every
    nonzero column runs exactly that many iterations and ``tol`` is unused.
    ``apply_M0`` is the mean-value preconditioner (one V-cycle).
    Returns ``(X, iters)`` with the per-column iteration counts.
    """
    n, w = B.shape
    X = np.zeros((n, w))
    iters = np.zeros(w, dtype=np.int64)
    cap = fixed_iters if fixed_iters > 0 else maxit
    for s in range(w):
        b = B[:, s].astype(np.float64)
        bb = float(b @ b)
        if bb == 0.0:
            continue
        x = np.zeros(n)
        r = b.copy()
        z = apply_M0(r)
        rho = float(r @ z)
        p = z.copy()
        for it in range(1, cap + 1):
            q = apply_A0(p)
            alpha = rho / float(p @ q)
            x += alpha * p
            r -= alpha * q
            iters[s] = it
            if fixed_iters == 0 and float(r @ r) <= tol * tol * bb:
                break
            if it == cap:
                break
            z = apply_M0(r)
            rho_new = float(r @ z)
            beta = rho_new / rho
            rho = rho_new
            p = z + beta * p
        X[:, s] = x
    return X, iters
