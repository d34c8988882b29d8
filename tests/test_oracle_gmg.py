"""Pins of the oracle's multigrid pieces: bilinear interpolation is exact,
Galerkin coarse operators equal the rediscretised coarse Q1 matrix, and the
V-cycle is a symmetric, positive definite, h-independent contraction."""
import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator

import sg_inputs as S
from oracle import gmg, sg_operator as so


@pytest.mark.parametrize("ne", [4, 8, 16])
def test_prolongation_is_bilinear_interpolation(ne):
    """P applied to coarse nodal values equals the piecewise bilinear
    interpolant (zero on the boundary) evaluated at the fine nodes."""
    rng = np.random.default_rng(ne)
    nc = ne // 2
    vals = np.zeros((nc + 1, nc + 1))                       # [y, x] incl. boundary zeros
    vals[1:nc, 1:nc] = rng.standard_normal((nc - 1, nc - 1))
    xs = np.linspace(0, 1, nc + 1)
    interp = RegularGridInterpolator((xs, xs), vals, method="linear")
    fx = np.linspace(0, 1, ne + 1)[1:ne]
    Y, X = np.meshgrid(fx, fx, indexing="ij")
    want = interp(np.stack([Y.ravel(), X.ravel()], axis=1))
    got = gmg.prolongation(ne) @ vals[1:nc, 1:nc].ravel()
    assert np.abs(got - want).max() < 1e-14


@pytest.mark.parametrize("ne", [8, 16, 32])
def test_galerkin_coarse_operator_is_coarse_q1_matrix(ne):
    """Nested Q1 spaces and exact quadrature: P^T A_h P = A_2h for the
    constant-coefficient mean matrix."""
    fine = S.make_problem(ne, 1, 0.1, 0.5, a_mean=1.3)
    coarse = S.make_problem(ne // 2, 1, 0.1, 0.5, a_mean=1.3)
    A0 = so.kl_matrices(fine.rowptr, fine.colidx, fine.vals)[0]
    Ac = so.kl_matrices(coarse.rowptr, coarse.colidx, coarse.vals)[0]
    lv = gmg.hierarchy(A0, ne)
    assert abs(lv[1].A - Ac).max() < 1e-13
    assert lv[-1].A.shape == (1, 1)


def test_vcycle_symmetric_positive_definite():
    ne = 8
    prob = S.make_problem(ne, 1, 0.1, 0.5)
    A0 = so.kl_matrices(prob.rowptr, prob.colidx, prob.vals)[0]
    lv = gmg.hierarchy(A0, ne)
    V = gmg.vcycle(lv, np.eye(prob.n))
    assert np.abs(V - V.T).max() < 1e-13
    assert np.linalg.eigvalsh(0.5 * (V + V.T))[0] > 0


@pytest.mark.parametrize("ne", [16, 32, 64])
def test_vcycle_contraction_h_independent(ne):
    prob = S.make_problem(ne, 1, 0.1, 0.5)
    A0 = so.kl_matrices(prob.rowptr, prob.colidx, prob.vals)[0]
    lv = gmg.hierarchy(A0, ne)
    x = np.random.default_rng(0).standard_normal(prob.n)
    for _ in range(25):
        y = x - gmg.vcycle(lv, A0 @ x)
        rate = np.linalg.norm(y) / np.linalg.norm(x)
        x = y / np.linalg.norm(y)
    assert rate < 0.15


def test_vcycle_columns_independent():
    ne = 16
    prob = S.make_problem(ne, 1, 0.1, 0.5)
    A0 = so.kl_matrices(prob.rowptr, prob.colidx, prob.vals)[0]
    lv = gmg.hierarchy(A0, ne)
    B = S.random_block(prob.n, 3, seed=4)
    Xb = gmg.vcycle(lv, B)
    for s in range(3):
        assert np.abs(Xb[:, s] - gmg.vcycle(lv, B[:, s])).max() < 1e-15


@pytest.mark.parametrize("ne,nu,omega,coef", [(8, 2, 0.8, "kl"), (16, 1, 0.7, "kl"), (16, 3, 0.6, "kl"),
                                             (8, 2, 0.8, "lognormal")])
def test_vcycle_equals_error_propagation_recursion(ne, nu, omega, coef):
    """The V-cycle as a matrix, from the textbook recursion of its error
    propagation rather than the procedure: with the damped Jacobi operator
    S_g = I - omega D_g^{-1} A_g, nu smoothing steps on each side of the coarse
    correction and the next grid's cycle E_{g+1} standing in for its exact
    solve, E_g = S_g^nu (I - P_g (I - E_{g+1}) A_{g+1}^{-1} P_g^T A_g) S_g^nu,
    E = 0 on the coarsest grid (solved exactly), and the cycle is
    V_g = (I - E_g) A_g^{-1}. The lognormal case's mean matrix has a
    spatially varying coefficient, hence a varying diagonal on every grid."""
    if coef == "kl":
        prob = S.make_problem(ne, 2, 0.3, 0.5)
    else:
        prob = S.make_lognormal_problem(ne, 2, 1.0, 0.5, 2)
    A0 = so.kl_matrices(prob.rowptr, prob.colidx, prob.vals)[0]
    lv = gmg.hierarchy(A0, ne)

    def E(g):
        Ag = lv[g].A.toarray()
        if g == len(lv) - 1:
            return np.zeros_like(Ag)
        Sg = np.eye(Ag.shape[0]) - omega * (Ag / np.diag(Ag)[:, None])
        Pg = lv[g].P.toarray()
        Ac = lv[g + 1].A.toarray()
        cgc = np.eye(Ag.shape[0]) - Pg @ (np.eye(Ac.shape[0]) - E(g + 1)) @ np.linalg.solve(Ac, Pg.T @ Ag)
        Sn = np.linalg.matrix_power(Sg, nu)
        return Sn @ cgc @ Sn

    Ad = A0.toarray()
    V_ref = (np.eye(prob.n) - E(0)) @ np.linalg.inv(Ad)
    V = gmg.vcycle(lv, np.eye(prob.n), nu=nu, omega=omega)
    assert np.abs(V - V_ref).max() <= 1e-11 * np.abs(V_ref).max()
