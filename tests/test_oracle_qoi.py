"""Pin of the oracle's adjoint gradient against central finite differences."""
import numpy as np
import pytest

import sg_inputs as S
from oracle import chaos, qoi, sg_operator as so


def _solve(ne, M, p, sigma, corr, a_mean, scale):
    prob = S.make_problem(ne, M, sigma, corr, a_mean=a_mean, sqrt_lambda_scale=scale)
    A = so.kl_matrices(prob.rowptr, prob.colidx, prob.vals)
    G = chaos.g_matrices(M, p)
    F = S.make_rhs(prob, p)
    U = so.direct_solve(A, G, F)
    import scipy.sparse as sp
    Mh = sp.csr_matrix((prob.mass, prob.colidx, prob.rowptr), shape=(prob.n, prob.n))
    return prob, A, G, U, Mh


def test_mass_matrix_integrates_constants():
    # sum over all nodes of the consistent mass is the area; on the interior
    # block it is the integral of (sum of interior hats)^2 -- check u = 1 on a
    # fine grid approaches 1
    prob = S.make_problem(64, 1, 0.1, 0.5)
    import scipy.sparse as sp
    Mh = sp.csr_matrix((prob.mass, prob.colidx, prob.rowptr), shape=(prob.n, prob.n))
    one = np.ones(prob.n)
    assert one @ (Mh @ one) == pytest.approx(1.0, abs=4.0 / 64)


def test_adjoint_gradient_matches_central_differences():
    ne, M, p, corr = 8, 2, 2, 0.6
    sigma, a_mean = 0.2, 1.1
    scale = np.array([1.0, 1.0])
    prob, A, G, U, Mh = _solve(ne, M, p, sigma, corr, a_mean, scale)
    Lam = so.direct_solve(A, G, 2.0 * (Mh @ U))
    g = qoi.qoi_grad(A, G, U, Lam, a_mean, sigma, prob.sqrt_lambda)
    s0 = prob.sqrt_lambda / scale
    h = 1e-6

    def Q(sig=sigma, am=a_mean, sc=scale):
        _, _, _, Uh, Mhh = _solve(ne, M, p, sig, corr, am, sc)
        return qoi.qoi(Uh, Mhh)

    fd = [(Q(am=a_mean + h) - Q(am=a_mean - h)) / (2 * h),
          (Q(sig=sigma + h) - Q(sig=sigma - h)) / (2 * h)]
    for k in range(M):
        e = np.zeros(M); e[k] = h
        # d/d s_k = (d/d scale_k) / s0_k
        fd.append((Q(sc=scale + e) - Q(sc=scale - e)) / (2 * h) / s0[k])
    fd = np.array(fd)
    assert np.abs(g - fd).max() <= 1e-6 * np.abs(fd).max()
