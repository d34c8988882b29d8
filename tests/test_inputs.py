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


def _q1_entry(ne, kappa, i, j, dx, dy, npts=2):
    """int kappa grad N_r . grad N_c over the unit square for the interior
    nodes r = (i, j) and c = (i + dx, j + dy) of the ne x ne Q1 grid, by
    npts x npts Gauss-Legendre quadrature on every element of the common
    support, with the bilinear hats written out: N(x, y) = t(x) t(y) with
    t(s) = 1 - |s - s_node| / h."""
    from numpy.polynomial import legendre as Leg
    h = 1.0 / ne
    t, w = Leg.leggauss(npts)
    tot = 0.0
    for ex in set((i - 1, i)) & set((i + dx - 1, i + dx)):
        for ey in set((j - 1, j)) & set((j + dy - 1, j + dy)):
            X, Y = np.meshgrid((ex + (t + 1) / 2) * h, (ey + (t + 1) / 2) * h, indexing="ij")
            W = np.outer(w, w) * h * h / 4

            def grad(a, b):
                sx, sy = X - a * h, Y - b * h
                hx, hy = 1 - np.abs(sx) / h, 1 - np.abs(sy) / h
                return -np.sign(sx) / h * hy, -np.sign(sy) / h * hx

            gr, gc = grad(i, j), grad(i + dx, j + dy)
            tot += float(np.sum(W * kappa(X, Y) * (gr[0] * gc[0] + gr[1] * gc[1])))
    return tot


def test_kl_stiffness_matrices_match_direct_integration():
    """Eq. (global-system): A_k = sigma s_k int phi_k grad N_r . grad N_c with
    phi_k(x, y) = e_a(x) e_b(y) the k-th 2-D KL pair and s_k = sqrt(lambda_k),
    and A_0 = a_mean int grad N_r . grad N_c: every entry of a few rows against
    the integral written out here in physical coordinates with the generator's
    quadrature (2 x 2 Gauss points per element), so the two agree to rounding;
    with 6 x 6 points they agree to the quadrature error (below 1 %)."""
    ne, M, sigma, L, a_mean = 8, 4, 0.3, 0.5, 1.7
    prob = S.make_problem(ne, M, sigma, L, a_mean=a_mean)
    kl = S.kl_2d(L, M)
    assert np.allclose(prob.sqrt_lambda, [math.sqrt(lam) for lam, _, _ in kl], rtol=0, atol=1e-15)
    assert any(mx is not my for _, mx, my in kl)          # some phi_k not symmetric in x and y
    m = ne - 1
    for (i, j) in [(1, 1), (3, 4), (6, 2)]:
        r = (j - 1) * m + (i - 1)
        for k in range(M + 1):
            if k == 0:
                kap = lambda X, Y: a_mean + 0 * X
            else:
                lam, mx, my = kl[k - 1]
                kap = lambda X, Y, lam=lam, mx=mx, my=my: sigma * math.sqrt(lam) * S.eval_kl_1d(mx, X) * S.eval_kl_1d(my, Y)
            got = {int(c): prob.vals[e, k] for e, c in zip(range(prob.rowptr[r], prob.rowptr[r + 1]),
                                                          prob.colidx[prob.rowptr[r]:prob.rowptr[r + 1]])}
            want = {}
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if 1 <= i + dx <= m and 1 <= j + dy <= m:
                        want[(j + dy - 1) * m + (i + dx - 1)] = _q1_entry(ne, kap, i, j, dx, dy)
            assert set(got) == set(want)
            scale = max(abs(v) for v in want.values())
            for c in want:
                assert abs(got[c] - want[c]) <= 1e-13 * scale, (i, j, k, c, got[c], want[c])
                fine = _q1_entry(ne, kap, i, j, c % m + 1 - i, c // m + 1 - j, npts=6)
                assert abs(got[c] - fine) <= 1e-2 * scale, (i, j, k, c, got[c], fine)


def test_lognormal_matrices_expand_the_stiffness_of_exp_g():
    """Sec. 6, lognormal case: sum_i A_i psi_i(xi), with the generator's gPC
    matrices up to degree q, approaches the stiffness matrix of the coefficient
    exp(g(x, xi)) itself, g = mu_g + sigma_g sum_k s_k phi_k(x) xi_k with
    sigma_g^2 = ln(1 + CoV^2) and mu_g = -sigma_g^2 / 2 (mean of exp(g) one),
    assembled here entry by entry by direct integration with the generator's
    2 x 2 Gauss points per element; what remains is the truncation of the
    expansion at degree q."""
    from numpy.polynomial import hermite_e as He
    ne, M, cov, L, q = 4, 2, 0.8, 0.5, 12
    prob = S.make_lognormal_problem(ne, M, cov, L, q)
    sig2 = math.log(1 + cov * cov)
    kl = S.kl_2d(L, M)
    xi = np.array([0.7, -1.1])

    def kap(X, Y):
        g = -0.5 * sig2 + 0.0 * X
        for k, (lam, mx, my) in enumerate(kl):
            g = g + math.sqrt(sig2) * math.sqrt(lam) * S.eval_kl_1d(mx, X) * S.eval_kl_1d(my, Y) * xi[k]
        return np.exp(g)

    gam = S._graded_indices(M, q)
    assert prob.vals.shape[1] == len(gam)
    psi = np.array([np.prod([He.hermeval(xi[k], [0] * g[k] + [1]) / math.sqrt(math.factorial(g[k]))
                             for k in range(M)]) for g in gam])
    Axi = prob.vals @ psi
    m = ne - 1
    for (i, j) in [(1, 1), (2, 2), (3, 1)]:
        r = (j - 1) * m + (i - 1)
        scale = 0.0
        errs = []
        for e in range(prob.rowptr[r], prob.rowptr[r + 1]):
            c = int(prob.colidx[e])
            want = _q1_entry(ne, kap, i, j, c % m + 1 - i, c // m + 1 - j)
            scale = max(scale, abs(want))
            errs.append(abs(Axi[e] - want))
        assert max(errs) <= 1e-8 * scale, (i, j, max(errs) / scale)
