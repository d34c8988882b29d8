"""Variants of eq. (general-prec) (Sec. 5): Algorithm 1 with the D_l^{-1} of
the pre-correction (M_D^1) and/or of the post-correction (M_D^2 = M_D^3)
replaced by the mean-value preconditioner M_0 alone, against the oracle's
Algorithm 1 with the same substitutions; and whole solves with them."""
import numpy as np
import pytest

import sg_inputs as S
from oracle import gmg, hsc, krylov, sg_operator as so
from tests.gpu_common import oracle_rel_residual, problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1205_1864_gb300 as L
    return L


def _t(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _np(t):
    return t.double().cpu().numpy()


@pytest.mark.parametrize("md", [1, 2, 3])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_variant_matches_oracle(lib, md, prec):
    ne, M, p = 16, 3, 3
    prob, A, G, off = problem(ne, M, p)
    h = lib.SGProblem.from_inputs(prob, p)
    lv = gmg.hierarchy(A[0], ne)
    R = S.random_block(prob.n, h.P, seed=21)
    pcg = lambda l, X: krylov.pcg_columns(lambda v: A[0] @ v, X, lambda r: gmg.vcycle(lv, r), tol=0.0, maxit=4,
                                          fixed_iters=4)[0]
    vc = lambda l, X: gmg.vcycle(lv, X)
    ref = hsc.hsc_apply(A, G, off, R, dsolve=pcg, dsolve_pre=vc if md & 1 else pcg,
                        dsolve_post=vc if md & 2 else pcg)
    o = lib.prec_opts(precision=lib.SG_F64 if prec == "f64" else lib.SG_F32, inner_fixed_iters=4, md_m0=md)
    Z = _np(lib.hsc_precond_apply(h, _t(R), o))
    tol = 1e-10 if prec == "f64" else 2e-5
    assert np.abs(Z - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("md", [0, 1, 2, 3])
def test_variant_solves(lib, md):
    """Each variant used as the preconditioner of flexible CG to 1e-8: the
    oracle's FP64 residual of the solution; Algorithm 1 itself (md = 0) needs
    the fewest iterations."""
    prob, A, G, off = problem(32, 4, 3, sigma=0.3)
    h = lib.SGProblem.from_inputs(prob, 3)
    F = S.make_rhs(prob, 3)
    o = lib.solve_opts(lib.prec_opts(precision=lib.SG_F32, md_m0=md), precond=lib.SG_PREC_HSC, tol=1e-8, maxit=500)
    U, st = lib.sg_solve(h, _t(F), o)
    assert oracle_rel_residual(A, G, F, _np(U)) <= 1.5e-8
    _, st0 = lib.sg_solve(h, _t(F), lib.solve_opts(lib.prec_opts(precision=lib.SG_F32), precond=lib.SG_PREC_HSC,
                                                    tol=1e-8))
    assert st0.iterations <= st.iterations
