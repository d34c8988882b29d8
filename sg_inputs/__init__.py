"""Seeded synthetic inputs for the stochastic Galerkin (SG) diffusion problem.

This module builds the *inputs* of the solve, and nothing of the solve
itself. The oracle (``oracle/``), the tests and the benchmark all call it; the
CUDA library never does. What it produces is what the paper's problem
statement feeds the solver (Sec. 2, eq. (model-1)-(model-2), (KL-expansion),
(cov), (global-system)):

* the Q1 finite-element mesh of the unit square ``[0,1]^2`` with ``ne x ne``
  elements, homogeneous Dirichlet nodes eliminated, interior nodes numbered
  lexicographically with ``x`` fastest;
* the truncated Karhunen-Loeve (KL) expansion of the coefficient
  ``a(x, xi) = a_mean + sigma * sum_k s_k phi_k(x) xi_k`` for the separable
  exponential covariance with the L1 norm, eq. (cov), ``s_k = sqrt(lambda_k)``;
* the KL stiffness matrices ``A_0..A_M`` (eq. (global-system): the paper's
  ``K_i``) on one shared CSR pattern, values stored ``[nnz][M+1]``;
* the load vector ``f_0`` for ``f = 1`` and the consistent Q1 mass matrix
  (used by the quantity of interest ``Q = E[int u^2]``);
* seeded draws for the batched and gradient workloads, and seeded random
  coefficient blocks for operator tests.

Readings of the paper used here (the paper is silent or garbled on these):
the random variables are ``xi_k ~ U(-sqrt3, sqrt3)`` (zero mean, unit
variance), so that CoV = sigma (Sec. 6); KL eigenpairs are the closed-form
1-D pairs of ``exp(-|s-t|/L)`` on ``[0,1]`` multiplied in 2-D and sorted by
``lambda`` descending, ties broken by ``(i+j, i)`` ascending; element
integrals use 2x2 Gauss quadrature.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np
from scipy.optimize import brentq

__all__ = [
    "kl_1d", "kl_2d", "Problem", "make_problem", "make_rhs", "random_block",
    "CONFIGS", "draw_batch_configs", "draw_grad_params", "chaos_count", "make_unit_problem", "theta_of",
    "make_lognormal_problem",
]


# ---------------------------------------------------------------------------
# Karhunen-Loeve expansion of exp(-|s-t|/L) on [0,1]  (Sec. 2, eq. (cov))
# ---------------------------------------------------------------------------

def kl_1d(corr_len: float, nterms: int):
    """Leading ``nterms`` eigenpairs of the kernel ``exp(-|s-t|/L)`` on [0,1].

    The kernel is shifted to ``[-a, a]`` with ``a = 1/2`` and ``c = 1/L``.
    Even modes ``cos(w t)`` solve ``c cos(wa) - w sin(wa) = 0`` with one root
    in each ``(i pi/a, (i+1/2) pi/a)``; odd modes ``sin(w t)`` solve
    ``w cos(wa) + c sin(wa) = 0`` with one root in each
    ``((i-1/2) pi/a, i pi/a)``. The eigenvalue is ``2c / (w^2 + c^2)``.

    Returns a list of ``(lam, w, parity, norm)`` sorted by ``lam`` descending,
    where the eigenfunction is ``norm * cos(w (t-1/2))`` for parity 0 and
    ``norm * sin(w (t-1/2))`` for parity 1, normalised in ``L2(0,1)``.
    """
    a = 0.5
    c = 1.0 / corr_len
    out = []
    i = 0
    eps = 1e-12
    while len(out) < nterms:
        # even root in (i pi / a, (i + 1/2) pi / a)
        lo, hi = i * math.pi / a + eps, (i + 0.5) * math.pi / a - eps
        w = brentq(lambda w: c * math.cos(w * a) - w * math.sin(w * a), lo, hi, xtol=1e-15, rtol=1e-15)
        nrm = 1.0 / math.sqrt(a + math.sin(2 * w * a) / (2 * w))
        out.append((2 * c / (w * w + c * c), w, 0, nrm))
        if len(out) >= nterms:
            break
        # odd root in ((i + 1/2) pi / a, (i + 1) pi / a)
        lo, hi = (i + 0.5) * math.pi / a + eps, (i + 1) * math.pi / a - eps
        w = brentq(lambda w: w * math.cos(w * a) + c * math.sin(w * a), lo, hi, xtol=1e-15, rtol=1e-15)
        nrm = 1.0 / math.sqrt(a - math.sin(2 * w * a) / (2 * w))
        out.append((2 * c / (w * w + c * c), w, 1, nrm))
        i += 1
    out.sort(key=lambda t: -t[0])
    return out[:nterms]


def eval_kl_1d(mode, t):
    lam, w, parity, nrm = mode
    s = np.asarray(t, dtype=np.float64) - 0.5
    return nrm * (np.cos(w * s) if parity == 0 else np.sin(w * s))


def kl_2d(corr_len: float, M: int):
    """Leading ``M`` 2-D eigenpairs of the separable L1 exponential kernel.

    Products ``lambda_i lambda_j`` of the 1-D pairs, sorted by value
    descending; equal products are ordered by ``i + j`` then ``i``
    ascending. Returns ``[(lam, mode_x, mode_y)]``.
    """
    n1 = M + 2
    modes = kl_1d(corr_len, n1)
    pairs = []
    for i in range(n1):
        for j in range(n1):
            pairs.append((modes[i][0] * modes[j][0], i + j, i, j))
    pairs.sort(key=lambda t: (-round(t[0], 14), t[1], t[2]))
    return [(lam, modes[i], modes[j]) for lam, _, i, j in pairs[:M]]


# ---------------------------------------------------------------------------
# Q1 finite elements on the unit square with Dirichlet nodes eliminated
# ---------------------------------------------------------------------------

_G = 1.0 / math.sqrt(3.0)
_GP = [(-_G, -_G), (_G, -_G), (-_G, _G), (_G, _G)]     # 2x2 Gauss points, weight 1 each
_LOC = [(0, 0), (1, 0), (0, 1), (1, 1)]                # local node (a, b): x offset a, y offset b


def _shape(a, b, xi, eta):
    sa, sb = 2 * a - 1, 2 * b - 1
    return (1 + sa * xi) * (1 + sb * eta) / 4.0, sa * (1 + sb * eta) / 4.0, sb * (1 + sa * xi) / 4.0


def _element_tables():
    """B[g,p,q] = grad N_p . grad N_q (reference coords), Mm[g,p,q] = N_p N_q at Gauss point g."""
    B = np.zeros((4, 4, 4))
    Mm = np.zeros((4, 4, 4))
    for g, (xi, eta) in enumerate(_GP):
        vals = [_shape(a, b, xi, eta) for a, b in _LOC]
        for p in range(4):
            for q in range(4):
                B[g, p, q] = vals[p][1] * vals[q][1] + vals[p][2] * vals[q][2]
                Mm[g, p, q] = vals[p][0] * vals[q][0]
    return B, Mm


def _assemble_stencils(ne: int, kappa_g: np.ndarray, table: np.ndarray, scale: float):
    """Sum element matrices into per-node 9-point stencils.

    ``kappa_g`` has shape ``(ncoef, ne_y, ne_x, 4)`` (coefficient values at the
    Gauss points of every element). Returns ``S`` of shape
    ``(9, ncoef, ne+1, ne+1)`` indexed ``[slot, k, y, x]`` with slot
    ``(dy+1)*3 + (dx+1)`` for the column node ``(x+dx, y+dy)``.
    """
    ncoef = kappa_g.shape[0]
    S = np.zeros((9, ncoef, ne + 1, ne + 1))
    tab = table.reshape(4, 16) * scale
    ke = np.empty((ne * ne, 16))
    for k in range(ncoef):
        np.matmul(kappa_g[k].reshape(-1, 4), tab, out=ke)
        ke3 = ke.reshape(ne, ne, 16)
        for p, (ap, bp) in enumerate(_LOC):
            for q, (aq, bq) in enumerate(_LOC):
                slot = (bq - bp + 1) * 3 + (aq - ap + 1)
                S[slot, k, bp:bp + ne, ap:ap + ne] += ke3[:, :, p * 4 + q]
    return S


def _interior_csr(ne: int, S: np.ndarray):
    """CSR (rowptr, colidx, vals[nnz][ncoef]) of the interior rows of stencils S."""
    m = ne - 1
    n = m * m
    ys, xs = np.meshgrid(np.arange(1, ne), np.arange(1, ne), indexing="ij")
    ys = ys.ravel(); xs = xs.ravel()
    cols, vals, valid = [], [], []
    for slot in range(9):
        dy, dx = slot // 3 - 1, slot % 3 - 1
        cy, cx = ys + dy, xs + dx
        ok = (cy >= 1) & (cy <= ne - 1) & (cx >= 1) & (cx <= ne - 1)
        valid.append(ok)
        cols.append((cy - 1) * m + (cx - 1))
        vals.append(S[slot][:, ys, xs].T)             # (n, ncoef)
    valid = np.stack(valid, axis=1)                    # (n, 9)
    cols = np.stack(cols, axis=1)
    vals = np.stack(vals, axis=1)                      # (n, 9, ncoef)
    counts = valid.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int32)
    rowptr[1:] = np.cumsum(counts)
    colidx = cols[valid].astype(np.int32)
    v = vals[valid]                                    # (nnz, ncoef), row-major, slots ascending
    return rowptr, colidx, np.ascontiguousarray(v)


@dataclasses.dataclass
class Problem:
    """One SG problem: shared CSR pattern, values ``[nnz][M+1]``, load, mass."""
    ne: int
    M: int
    sigma: float
    corr_len: float
    a_mean: float
    sqrt_lambda: np.ndarray      # (M,) s_k = sqrt(lambda_k) as used (after any scaling)
    rowptr: np.ndarray           # (n+1,) int32
    colidx: np.ndarray           # (nnz,) int32
    vals: np.ndarray             # (nnz, M+1) float64: A_0 .. A_M on the shared pattern
    mass: np.ndarray             # (nnz,) float64: consistent Q1 mass matrix
    f0: np.ndarray               # (n,) float64: load vector of f = 1
    coef_degree: int = -1        # -1: linear KL expansion (vals has M+1 terms); q >= 0: gPC expansion of
                                 # the coefficient to total degree q (vals has C(M+q, M) terms, graded order)

    @property
    def n(self) -> int:
        return int(self.rowptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.colidx.shape[0])


def make_problem(ne: int, M: int, sigma: float, corr_len: float, a_mean: float = 1.0,
                 sqrt_lambda_scale: Optional[Sequence[float]] = None) -> Problem:
    """Assemble the KL stiffness matrices of ``a(x,xi)`` on an ``ne x ne`` Q1 grid.

    ``A_0 = a_mean * L_h`` (the mean-value problem, Sec. 3 eq.
    (mean-value-problem)) and ``A_k = sigma * s_k * Phi_k`` with
    ``(Phi_k)_{rc} = int phi_k grad N_r . grad N_c`` for ``k = 1..M``
    (the paper's ``K_i`` of eq. (global-system)). ``sqrt_lambda_scale``
    multiplies each ``s_k`` (used by the gradient workload).
    """
    if ne < 2:
        raise ValueError("ne must be >= 2")
    h = 1.0 / ne
    kl = kl_2d(corr_len, M) if M > 0 else []
    s = np.array([math.sqrt(lam) for lam, _, _ in kl], dtype=np.float64)
    if sqrt_lambda_scale is not None:
        s = s * np.asarray(sqrt_lambda_scale, dtype=np.float64)
    # Gauss point coordinates per element
    ex = np.arange(ne)
    gx = np.stack([(ex + (1 + xi) / 2) * h for xi, _ in _GP], axis=-1)   # (ne, 4) x of each gp
    gy = np.stack([(ex + (1 + eta) / 2) * h for _, eta in _GP], axis=-1)
    kappa = np.empty((M + 1, ne, ne, 4))
    kappa[0] = a_mean
    for k, (lam, mx, my) in enumerate(kl, start=1):
        fx = eval_kl_1d(mx, gx)                                          # (ne_x, 4)
        fy = eval_kl_1d(my, gy)                                          # (ne_y, 4)
        kappa[k] = sigma * s[k - 1] * fy[:, None, :] * fx[None, :, :]
    B, Mm = _element_tables()
    S = _assemble_stencils(ne, kappa, B, 1.0)
    rowptr, colidx, vals = _interior_csr(ne, S)
    Sm = _assemble_stencils(ne, np.ones((1, ne, ne, 4)), Mm, h * h / 4.0)
    _, _, mass = _interior_csr(ne, Sm)
    n = (ne - 1) ** 2
    f0 = np.full(n, h * h)
    return Problem(ne=ne, M=M, sigma=sigma, corr_len=corr_len, a_mean=a_mean, sqrt_lambda=s,
                   rowptr=rowptr, colidx=colidx, vals=vals, mass=mass[:, 0].copy(), f0=f0)


def _graded_indices(M: int, q: int) -> List[tuple]:
    """Multi-indices of total degree <= q: degrees ascending, descending
    lexicographic order inside a degree (the chaos order of the solver)."""
    def desc(d, m):
        if m == 1:
            yield (d,)
            return
        for a in range(d, -1, -1):
            for rest in desc(d - a, m - 1):
                yield (a,) + rest
    out = []
    for d in range(q + 1):
        out.extend(desc(d, M) if M > 0 else ([()] if d == 0 else []))
    return out


def make_lognormal_problem(ne: int, M: int, cov: float, corr_len: float, q: int) -> Problem:
    """Stiffness matrices of the gPC expansion of a lognormal coefficient
    (Sec. 6, second set of experiments; Remark K-L).

    ``k(x, xi) = exp(g(x, xi))`` with the Gaussian field
    ``g = mu_g + sigma_g sum_k s_k phi_k(x) xi_k``, ``xi_k ~ N(0,1)``, the same
    separable exponential-covariance KL pairs as the uniform case. Reading of
    the paper's "CoV = sigma_log / mu_log" (the mean and standard deviation of
    ``k`` itself, mean 1): ``sigma_g^2 = ln(1 + CoV^2)``, ``mu_g = -sigma_g^2/2``.
    Its expansion in normalised Hermite polynomials ``psi_gamma`` has the
    closed-form coefficients
    ``k_gamma(x) = exp(mu_g + sum_k a_k(x)^2 / 2) prod_k a_k(x)^gamma_k / sqrt(gamma_k!)``
    with ``a_k = sigma_g s_k phi_k`` (the generating function of Hermite
    polynomials). The expansion is kept to total degree ``q`` (the paper uses
    twice the degree of the solution); ``vals[:, i]`` is the stiffness matrix of
    ``k_gamma_i``, ``gamma_i`` in the graded chaos order.
    """
    if ne < 2:
        raise ValueError("ne must be >= 2")
    h = 1.0 / ne
    kl = kl_2d(corr_len, M) if M > 0 else []
    s = np.array([math.sqrt(lam) for lam, _, _ in kl], dtype=np.float64)
    sig2 = math.log(1.0 + cov * cov)
    sig_g, mu_g = math.sqrt(sig2), -0.5 * sig2
    ex = np.arange(ne)
    gx = np.stack([(ex + (1 + xi) / 2) * h for xi, _ in _GP], axis=-1)
    gy = np.stack([(ex + (1 + eta) / 2) * h for _, eta in _GP], axis=-1)
    a = np.empty((M, ne, ne, 4))
    for k, (lam, mx, my) in enumerate(kl):
        a[k] = sig_g * s[k] * eval_kl_1d(my, gy)[:, None, :] * eval_kl_1d(mx, gx)[None, :, :]
    mean = np.exp(mu_g + 0.5 * np.sum(a * a, axis=0)) if M > 0 else np.full((ne, ne, 4), math.exp(mu_g))
    gammas = _graded_indices(M, q)
    kappa = np.empty((len(gammas), ne, ne, 4))
    for i, g in enumerate(gammas):
        v = mean.copy()
        for k, gk in enumerate(g):
            if gk:
                v *= a[k] ** gk / math.sqrt(math.factorial(gk))
        kappa[i] = v
    B, Mm = _element_tables()
    S = _assemble_stencils(ne, kappa, B, 1.0)
    rowptr, colidx, vals = _interior_csr(ne, S)
    Sm = _assemble_stencils(ne, np.ones((1, ne, ne, 4)), Mm, h * h / 4.0)
    _, _, mass = _interior_csr(ne, Sm)
    n = (ne - 1) ** 2
    return Problem(ne=ne, M=M, sigma=sig_g, corr_len=corr_len, a_mean=1.0, sqrt_lambda=s, rowptr=rowptr,
                   colidx=colidx, vals=vals, mass=mass[:, 0].copy(), f0=np.full(n, h * h), coef_degree=q)


def make_unit_problem(ne: int, M: int, corr_len: float) -> Problem:
    """KL matrices with unit parameters: A_0 = L_h (a_mean = 1) and
    A_k = Phi_k (sigma = 1, s_k = 1); a parameter set theta = (a_mean, sigma,
    s_1..s_M) then scales them as A_0 = a_mean L_h, A_k = sigma s_k Phi_k."""
    kl = kl_2d(corr_len, M) if M > 0 else []
    inv = [1.0 / math.sqrt(lam) for lam, _, _ in kl]
    return make_problem(ne, M, 1.0, corr_len, a_mean=1.0, sqrt_lambda_scale=inv if M > 0 else None)


def theta_of(prob: Problem) -> np.ndarray:
    """theta = (a_mean, sigma, s_1..s_M) of an assembled problem."""
    return np.concatenate([[prob.a_mean, prob.sigma], prob.sqrt_lambda])


def chaos_count(M: int, p: int) -> int:
    """Number of chaos polynomials of total degree <= p in M variables."""
    return math.comb(M + p, M)


def make_rhs(prob: Problem, p: int) -> np.ndarray:
    """SG right-hand side ``F`` (n x P, row-major, chaos index fastest).

    Only the degree-0 column is nonzero, since ``E[psi_j] = 0`` for j >= 1
    (Sec. 2, the definition of ``f_k`` below eq. (global-system)).
    """
    P = chaos_count(prob.M, p)
    F = np.zeros((prob.n, P))
    F[:, 0] = prob.f0
    return F


def random_block(n: int, P: int, seed: int = 1205, dtype=np.float64) -> np.ndarray:
    """Seeded uniform(-1, 1) coefficient block of shape (n, P)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1.0, 1.0, size=(n, P)).astype(dtype)


# ---------------------------------------------------------------------------
# Workloads: the five synthetic configurations and their seeded draws
# ---------------------------------------------------------------------------

CONFIGS = {
    # plain method, all FP64, 16x16 grid, M=3, p=3
    "cfg1_fp64_16x16_M3_p3": dict(ne=16, M=3, p=3, sigma=0.2, corr_len=0.5),
    # single large mixed-precision solve, 128x128 grid, M=6, p=4
    "cfg2_mixed_128x128_M6_p4": dict(ne=128, M=6, p=4, sigma=0.3, corr_len=1.0),
    # gradient workload, 64x64 grid, M=4, p=3 (sigma, a_mean, s_k drawn per set)
    "cfg4_grad_64x64_M4_p3": dict(ne=64, M=4, p=3, sigma=0.2, corr_len=0.5),
    # largest single system, 512x512 grid, M=10, p=4
    "cfg5_large_512x512_M10_p4": dict(ne=512, M=10, p=4, sigma=0.25, corr_len=0.5),
}


def draw_batch_configs(count: int = 64, seed: int = 1864,
                       meshes: Sequence[int] = (32, 64, 128, 256)) -> List[dict]:
    """Seeded draws for the batched workload: per system, in this order,
    mesh from ``meshes``, M in 2..8, p in 2..4, sigma in [0.1, 0.3],
    correlation length in [0.3, 1.5]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        ne = int(meshes[int(rng.integers(0, len(meshes)))])
        M = int(rng.integers(2, 9))
        p = int(rng.integers(2, 5))
        sigma = float(rng.uniform(0.1, 0.3))
        corr = float(rng.uniform(0.3, 1.5))
        out.append(dict(ne=ne, M=M, p=p, sigma=sigma, corr_len=corr))
    return out


def draw_grad_params(M: int, count: int = 16, seed: int = 4) -> List[dict]:
    """Seeded parameter sets for the gradient workload: sigma in [0.1, 0.25],
    a_mean in [0.8, 1.2], each s_k scaled by a factor in [0.9, 1.1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        sigma = float(rng.uniform(0.1, 0.25))
        a_mean = float(rng.uniform(0.8, 1.2))
        scale = rng.uniform(0.9, 1.1, size=M)
        out.append(dict(sigma=sigma, a_mean=a_mean, sqrt_lambda_scale=scale))
    return out
