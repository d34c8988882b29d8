"""Pins of the seeded input generator: the KL closed form against a Nystrom
discretisation of eq. (int-eigproblem), and the Q1 assembly against the
textbook stencil."""
import math

import numpy as np
import pytest

import sg_inputs as S


@pytest.mark.parametrize("L", [0.3, 0.5, 1.0, 1.5])
def test_kl_1d_closed_form_matches_nystrom(L):
    m = 2000
    t = (np.arange(m) + 0.5) / m
    Kmat = np.exp(-np.abs(t[:, None] - t[None, :]) / L) / m
    ev = np.sort(np.linalg.eigvalsh(Kmat))[::-1][:6]
    modes = S.kl_1d(L, 6)
    lam = np.array([md[0] for md in modes])
    assert np.allclose(lam, ev, rtol=2e-4)
    # eigenfunctions orthonormal in L2(0,1)
    F = np.stack([S.eval_kl_1d(md, t) for md in modes])
    assert np.allclose(F @ F.T / m, np.eye(6), atol=1e-5)
    # trace of the unit-variance kernel on [0,1] is 1
    assert sum(md[0] for md in S.kl_1d(L, 400)) == pytest.approx(1.0, abs=0.01 * L + 2e-3)


def test_kl_2d_products_sorted():
    kl = S.kl_2d(0.5, 10)
    lam = [k[0] for k in kl]
    assert all(a >= b - 1e-15 for a, b in zip(lam, lam[1:]))
    assert lam[:4] == pytest.approx([0.3302, 0.1123, 0.1123, 0.0451], abs=5e-5)


def test_q1_mean_matrix_is_textbook_stencil():
    ne = 8
    prob = S.make_problem(ne, 2, 0.3, 0.5, a_mean=2.0)
    n = prob.n
    assert n == (ne - 1) ** 2
    # an interior row far from the boundary: 8/3 centre, -1/3 for 8 neighbours
    r = 3 * (ne - 1) + 3
    cols = prob.colidx[prob.rowptr[r]:prob.rowptr[r + 1]]
    vals = prob.vals[prob.rowptr[r]:prob.rowptr[r + 1], 0]
    assert len(cols) == 9
    assert np.allclose(np.sort(vals), 2.0 * np.array([-1 / 3] * 8 + [8 / 3]))
    # shared sorted pattern, symmetric values for every k
    import scipy.sparse as sp
    for k in range(3):
        A = sp.csr_matrix((prob.vals[:, k], prob.colidx, prob.rowptr), shape=(n, n))
        assert abs(A - A.T).max() < 1e-15
    for r in range(n):
        c = prob.colidx[prob.rowptr[r]:prob.rowptr[r + 1]]
        assert np.all(np.diff(c) > 0)
    assert np.allclose(prob.f0, 1.0 / ne ** 2)


def test_kl_stiffness_is_weighted_laplacian():
    """With a constant KL function the weighted stiffness is the Laplacian:
    checked through the bilinear form of a linear field (u = x) on interior
    rows away from the boundary, where -div(grad x) = 0."""
    ne = 16
    prob = S.make_problem(ne, 1, 0.4, 0.5)
    n = prob.n
    import scipy.sparse as sp
    A1 = sp.csr_matrix((prob.vals[:, 1], prob.colidx, prob.rowptr), shape=(n, n))
    xs = np.tile(np.arange(1, ne) / ne, ne - 1)
    # interior rows whose full stencil is interior: (A_1 x)_r = int phi_1 grad x . grad N_r
    # integrates d(phi_1)/dx * N_r ... sign-indefinite but small; the Laplacian case is exact 0
    A0 = sp.csr_matrix((prob.vals[:, 0], prob.colidx, prob.rowptr), shape=(n, n))
    y = A0 @ xs
    inner = [(j - 1) * (ne - 1) + (i - 1) for j in range(2, ne - 1) for i in range(2, ne - 1)]
    assert np.abs(y[inner]).max() < 1e-13


def test_draws_seeded_and_in_range():
    a = S.draw_batch_configs(64)
    b = S.draw_batch_configs(64)
    assert a == b
    for c in a:
        assert c["ne"] in (32, 64, 128, 256) and 2 <= c["M"] <= 8 and 2 <= c["p"] <= 4
        assert 0.1 <= c["sigma"] <= 0.3 and 0.3 <= c["corr_len"] <= 1.5
    g = S.draw_grad_params(4, 16)
    assert len(g) == 16 and all(0.1 <= d["sigma"] <= 0.25 for d in g)


def test_lognormal_gpc_coefficients_reproduce_the_field():
    """The closed-form gPC coefficients of the lognormal coefficient: at an
    interior Gauss point, sum_i k_i(x) psi_i(xi) approaches exp(g(x, xi)) as
    the expansion degree grows, and k_0 is the mean of exp(g)."""
    import math as _m

    from numpy.polynomial import hermite_e as He
    ne, M, cov, L = 4, 2, 1.0, 0.5
    sig2 = _m.log(1 + cov * cov)
    kl = S.kl_2d(L, M)
    hx = 1.0 / ne
    g0 = (1 - 1 / _m.sqrt(3)) / 2 * hx                      # first Gauss point of the first element
    a = np.array([_m.sqrt(sig2) * _m.sqrt(lam) * S.eval_kl_1d(mx, g0) * S.eval_kl_1d(my, g0) for lam, mx, my in kl])
    rng = np.random.default_rng(3)
    xi = rng.standard_normal(M) * 0.8
    exact = _m.exp(-0.5 * sig2 + float(a @ xi))
    assert S._graded_indices(M, 1) == [(0, 0), (1, 0), (0, 1)]
    errs = []
    for q in (2, 6, 12):
        gam = S._graded_indices(M, q)
        mean = _m.exp(-0.5 * sig2 + 0.5 * float(a @ a))
        tot = 0.0
        for g in gam:
            ki = mean * np.prod([a[k] ** g[k] / _m.sqrt(_m.factorial(g[k])) for k in range(M)])
            psi = np.prod([He.hermeval(xi[k], [0] * g[k] + [1]) / _m.sqrt(_m.factorial(g[k])) for k in range(M)])
            tot += ki * psi
        errs.append(abs(tot - exact) / exact)
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-9
    prob = S.make_lognormal_problem(ne, M, cov, L, 4)
    assert prob.vals.shape[1] == _m.comb(M + 4, M) and prob.coef_degree == 4
    # the mean matrix is a stiffness matrix of a positive coefficient: symmetric, positive diagonal
    import scipy.sparse as sp
    A0 = sp.csr_matrix((prob.vals[:, 0], prob.colidx, prob.rowptr), shape=(prob.n, prob.n))
    assert abs(A0 - A0.T).max() < 1e-14 and np.all(A0.diagonal() > 0)
