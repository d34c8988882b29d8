"""Quantity of interest ``Q = E[int_D u^2]`` and its adjoint gradient (oracle;
test infrastructure only).

The paper has no gradient; this is the reading used by the build. With the
orthonormal chaos basis ``E[psi_j psi_l] = delta_jl``, so
``Q = sum_j u_j^T M_h u_j`` with the consistent Q1 mass matrix ``M_h``.
The SG matrix ``A(theta) = sum_k A_k(theta) (x) G_k`` is symmetric, so with
``A u = f`` and ``A lam = dQ/du = 2 (M_h (x) I) u``,
``dQ/dtheta = -lam^T (dA/dtheta) u = -sum_k <Lam, (dA_k/dtheta) U G_k^T>_F``.
Parameters: ``A_0 = a_mean L_h`` and ``A_k = sigma s_k Phi_k``, so
``dA_0/da_mean = A_0/a_mean``, ``dA_k/dsigma = A_k/sigma`` and
``dA_k/ds_k = A_k/s_k``.
"""
from __future__ import annotations

import numpy as np

from .sg_operator import sg_apply


def qoi(U: np.ndarray, Mh) -> float:
    """``Q = sum_j u_j^T M_h u_j``."""
    return float(np.sum(U * (Mh @ U)))


def k_resolved_products(A, G, U: np.ndarray, Lam: np.ndarray) -> np.ndarray:
    """``h_k = <Lam, A_k U G_k^T>_F`` for ``k = 0..M``."""
    return np.array([float(np.sum(Lam * sg_apply([Ak], [Gk], U))) for Ak, Gk in zip(A, G)])


def chain_weights(a_mean: float, sigma: float, s: np.ndarray) -> np.ndarray:
    """``W[theta][k] = -(d log A_k / d theta)`` for ``theta = (a_mean, sigma,
    s_1..s_M)`` so that ``dQ/dtheta = sum_k W[theta][k] h_k``."""
    M = len(s)
    W = np.zeros((M + 2, M + 1))
    W[0, 0] = -1.0 / a_mean
    W[1, 1:] = -1.0 / sigma
    for k in range(M):
        W[2 + k, 1 + k] = -1.0 / s[k]
    return W


def qoi_grad(A, G, U: np.ndarray, Lam: np.ndarray, a_mean: float, sigma: float, s: np.ndarray) -> np.ndarray:
    """``dQ/d(a_mean, sigma, s_1..s_M)`` from the forward and adjoint solutions."""
    return chain_weights(a_mean, sigma, s) @ k_resolved_products(A, G, U, Lam)
