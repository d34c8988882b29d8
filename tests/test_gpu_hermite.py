"""Hermite chaos (Gaussian xi, normalised probabilists' Hermite polynomials)
through the C ABI against the FP64 oracle: the triple products enter the SG
product and the level products, and the hierarchical Schur complement solve
applies unchanged because multiplying by xi_k still moves the degree by
exactly one (the Lemma of Sec. 3: D_l = I (x) A_0)."""
import numpy as np
import pytest

import sg_inputs as S
from oracle import chaos, sg_operator as so
from tests.gpu_common import TOL32, TOL64, abs_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1205_1864_gb300 as L
    return L


def _t(x, dtype=None):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype or torch.float64, device="cuda")


def _np(t):
    return t.double().cpu().numpy()


def _hermite(ne, M, p, sigma):
    prob = S.make_problem(ne, M, sigma, 0.6)
    A = so.kl_matrices(prob.rowptr, prob.colidx, prob.vals)
    G = chaos.g_matrices(M, p, family=chaos.HERMITE)
    _, off = chaos.multi_indices(M, p)
    return prob, A, G, off


@pytest.mark.parametrize("ne,M,p", [(16, 3, 3), (8, 2, 4)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_hermite_sg_apply_parity(lib, ne, M, p, prec):
    import torch
    prob, A, G, off = _hermite(ne, M, p, 0.1)
    h = lib.SGProblem.from_inputs(prob, p, family=lib.SG_HERMITE)
    U = S.random_block(prob.n, h.P, seed=11)
    dt = torch.float64 if prec == "f64" else torch.float32
    if prec == "f32":
        U = U.astype(np.float32).astype(np.float64)
    Y = _np(lib.sg_apply(h, _t(U, dt)))
    ref = so.sg_apply(A, G, U)
    tol = TOL64 if prec == "f64" else TOL32
    assert np.all(np.abs(Y - ref) <= tol * abs_bound(A, G, U) + 1e-300)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_hermite_hsc_solve_matches_direct_solve(lib, prec):
    prob, A, G, off = _hermite(16, 3, 3, 0.1)
    h = lib.SGProblem.from_inputs(prob, 3, family=lib.SG_HERMITE)
    F = S.make_rhs(prob, 3)
    ref = so.direct_solve(A, G, F)
    dt = lib.SG_F64 if prec == "f64" else lib.SG_F32
    U, st = lib.sg_solve(h, _t(F), lib.solve_opts(lib.prec_opts(precision=dt), precond=lib.SG_PREC_HSC,
                                                   tol=1e-13 if prec == "f64" else 1e-12))
    bound = 1e-10 if prec == "f64" else 1e-7
    assert np.abs(_np(U) - ref).max() <= bound * np.abs(ref).max()
    assert st.iterations < 30
