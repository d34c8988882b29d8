"""Pins of the oracle's chaos basis and triple products against closed forms,
brute-force quadrature and the block counts printed in the paper."""
import itertools
import math
import os

import numpy as np
import pytest
from numpy.polynomial import hermite_e as He
from numpy.polynomial import legendre as Leg

from oracle import chaos

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("M,p", [(1, 4), (2, 3), (3, 3), (4, 4), (6, 4), (10, 4), (8, 2)])
def test_multi_index_table_is_graded_complete_and_ordered(M, p):
    alpha, off = chaos.multi_indices(M, p)
    # eq. (gPC-u): (M+p)!/(M!p!) polynomials
    assert alpha.shape == (math.comb(M + p, M), M)
    assert chaos.chaos_count(M, p) == alpha.shape[0]
    assert off[-1] == alpha.shape[0]
    deg = alpha.sum(axis=1)
    for d in range(p + 1):
        blk = alpha[off[d]:off[d + 1]]
        assert np.all(blk.sum(axis=1) == d)
        assert blk.shape[0] == math.comb(M + d - 1, d)
        # strictly descending lexicographic inside the degree
        for a, b in zip(blk[:-1], blk[1:]):
            assert tuple(a) > tuple(b)
    assert np.all(np.diff(deg) >= 0)
    # every multi-index with |alpha| <= p is present exactly once
    full = {t for t in itertools.product(range(p + 1), repeat=M) if sum(t) <= p}
    assert {tuple(a) for a in alpha} == full
    if p >= 1:
        assert np.array_equal(alpha[off[1]:off[2]], np.eye(M, dtype=np.int64))


def _psi_1d(family, m, x):
    """Orthonormal 1-D polynomial of degree m built independently from numpy."""
    if family == chaos.LEGENDRE:
        c = np.zeros(m + 1); c[m] = 1
        return math.sqrt(2 * m + 1) * Leg.legval(x / math.sqrt(3.0), c)
    c = np.zeros(m + 1); c[m] = 1
    return He.hermeval(x, c) / math.sqrt(math.factorial(m))


def _quad_1d(family, npts):
    if family == chaos.LEGENDRE:
        t, w = Leg.leggauss(npts)          # uniform on [-1,1]: density 1/2
        return math.sqrt(3.0) * t, w / 2.0
    x, w = He.hermegauss(npts)              # weight exp(-x^2/2)
    return x, w / math.sqrt(2 * math.pi)


@pytest.mark.parametrize("family", [chaos.LEGENDRE, chaos.HERMITE])
@pytest.mark.parametrize("M,p", [(2, 3), (3, 2)])
def test_triple_products_match_brute_force_quadrature(family, M, p):
    """(G_k)_{jl} = E[xi_k psi_j psi_l] by tensor Gauss quadrature of the full
    M-dimensional integrand, with the polynomials evaluated from numpy."""
    alpha, _ = chaos.multi_indices(M, p)
    P = alpha.shape[0]
    x1, w1 = _quad_1d(family, p + 3)
    pts = np.array(list(itertools.product(x1, repeat=M)))
    wts = np.prod(np.array(list(itertools.product(w1, repeat=M))), axis=1)
    psi = np.ones((P, pts.shape[0]))
    for j in range(P):
        for i in range(M):
            psi[j] *= _psi_1d(family, alpha[j, i], pts[:, i])
    Gs = chaos.g_matrices(M, p, family)
    # orthonormality: E[psi_j psi_l] = delta_jl = G_0
    E0 = (psi * wts) @ psi.T
    assert np.allclose(E0, Gs[0].toarray(), atol=1e-12)
    for k in range(M):
        Ek = (psi * wts * pts[:, k]) @ psi.T
        assert np.allclose(Ek, Gs[k + 1].toarray(), atol=1e-12), k


def test_xi_is_first_order_chaos_polynomial():
    # psi_{e_k} = xi_k for both normalised families, so E[xi_k psi_0 psi_{e_k}] = 1
    for fam in (chaos.LEGENDRE, chaos.HERMITE):
        assert chaos.xi_triple_1d(0, fam) == pytest.approx(1.0, abs=1e-15)


@pytest.mark.parametrize("M,p", [(2, 3), (4, 4), (6, 4), (10, 4)])
def test_g_symmetric_and_lemma_diagonal_block(M, p):
    """Sec. 3 Lemma: the block d_l of c_P is diagonal, i.e. no G_k with k >= 1
    couples two chaos polynomials of the same degree."""
    _, off = chaos.multi_indices(M, p)
    Gs = chaos.g_matrices(M, p)
    for k, G in enumerate(Gs):
        assert abs(G - G.T).max() == 0
        if k == 0:
            continue
        for l in range(p + 1):
            assert Gs[k][off[l]:off[l + 1], off[l]:off[l + 1]].nnz == 0
        # linear KL couples degree d only with d +- 1
        for l1 in range(p + 1):
            for l2 in range(p + 1):
                if abs(l1 - l2) != 1:
                    assert Gs[k][off[l1]:off[l1 + 1], off[l2]:off[l2 + 1]].nnz == 0


def _read_table5():
    rows, fig = [], []
    with open(os.path.join(GOLDEN, "table5_block_counts.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if parts[0] == "fig1":
                fig.append(tuple(int(v) for v in parts[1:]))
            else:
                rows.append(tuple(int(v) for v in parts))
    return rows, fig


def test_block_counts_reproduce_table5_and_fig1():
    rows, fig = _read_table5()
    assert len(rows) == 8
    for NP, n_b, n_db, n_m, n_ds in rows:
        for M, p in ((NP, 4), (4, NP)):   # Table 5: either parameter varies, the other is 4
            c = chaos.block_counts(M, p)
            assert (c["n_b"], c["n_db"], c["n_m"], c["n_ds"]) == (n_b, n_db, n_m, n_ds), (M, p)
    for M, p, n_b in fig:
        assert chaos.block_counts(M, p)["n_b"] == n_b


@pytest.mark.parametrize("M", range(1, 11))
@pytest.mark.parametrize("p", range(1, 5))
def test_block_count_closed_forms(M, p):
    c = chaos.block_counts(M, p)
    assert c["n_db"] == math.comb(M + p, M)
    assert c["n_m"] == 2 * M * math.comb(M + p - 1, M)


def test_hermite_triple_products_against_quadrature():
    """The closed-form normalised Hermite triple products against Gauss-Hermite
    quadrature (probabilists' weight), all orders up to 8."""
    from numpy.polynomial import hermite_e as He
    x, w = He.hermegauss(40)
    w = w / np.sqrt(2 * np.pi)
    psi = [He.hermeval(x, [0] * m + [1]) / math.sqrt(math.factorial(m)) for m in range(9)]
    for a in range(9):
        for b in range(9):
            for c in range(9):
                ref = float(np.sum(w * psi[a] * psi[b] * psi[c]))
                assert chaos.hermite_triple_1d(a, b, c) == pytest.approx(ref, abs=1e-9 * max(1.0, abs(ref)))


@pytest.mark.parametrize("M,p", [(2, 3), (3, 2)])
def test_gpc_matrices_reduce_to_the_linear_expansion(M, p):
    """With the coefficient expanded to degree 1 the gPC matrices are the KL
    ones of the Hermite family: G_0 = I and G_{e_k} = E[xi_k psi_j psi_l]; for
    any degree each G_i is symmetric and couples j, l only when the degrees
    allow it (|alpha_j| - |alpha_l| <= |gamma_i| <= |alpha_j| + |alpha_l|)."""
    G1 = chaos.gpc_g_matrices(M, p, 1)
    Gk = chaos.g_matrices(M, p, chaos.HERMITE)
    assert len(G1) == len(Gk)
    for a, b in zip(G1, Gk):
        assert abs(a - b).max() < 1e-14
    Gq = chaos.gpc_g_matrices(M, p, 2 * p)
    alpha, _ = chaos.multi_indices(M, p)
    gamma, _ = chaos.multi_indices(M, 2 * p)
    for g, G in zip(gamma, Gq):
        assert abs(G - G.T).max() < 1e-14
        C = G.tocoo()
        for j, l in zip(C.row, C.col):
            dj, dl, dg = alpha[j].sum(), alpha[l].sum(), g.sum()
            assert abs(dj - dl) <= dg <= dj + dl


@pytest.mark.parametrize("M,p,q", [(2, 2, 4), (3, 1, 2), (1, 3, 6)])
def test_gpc_triple_products_match_brute_force_quadrature(M, p, q):
    """(G_i)_{jl} = E[psi_i psi_j psi_l] for every coefficient polynomial psi_i
    of total degree <= q (the lognormal case expands the coefficient to
    q = 2p), by tensor Gauss-Hermite quadrature of the M-dimensional integrand
    with the polynomials evaluated from numpy; the rule is exact for the
    integrand's degree q + 2p per coordinate."""
    alpha, _ = chaos.multi_indices(M, p)
    gamma, _ = chaos.multi_indices(M, q)
    Gq = chaos.gpc_g_matrices(M, p, q)
    assert len(Gq) == math.comb(M + q, M)
    x1, w1 = _quad_1d(chaos.HERMITE, p + q // 2 + 2)
    pts = np.array(list(itertools.product(x1, repeat=M)))
    wts = np.prod(np.array(list(itertools.product(w1, repeat=M))), axis=1)

    def table(idx):
        out = np.ones((idx.shape[0], pts.shape[0]))
        for j in range(idx.shape[0]):
            for i in range(M):
                out[j] *= _psi_1d(chaos.HERMITE, idx[j, i], pts[:, i])
        return out

    psi, phi = table(alpha), table(gamma)
    for i in range(gamma.shape[0]):
        E = (psi * wts * phi[i]) @ psi.T
        assert np.allclose(E, Gq[i].toarray(), rtol=0, atol=1e-10 * max(1.0, np.abs(E).max())), i
