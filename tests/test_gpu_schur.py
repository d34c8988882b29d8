"""The Schur-reduced outer system of Sec. 5 (eq. (global-Schur-system)) on
the GPU: the degree-p unknowns eliminated a priori, flexible CG on
S_{p-1} u_{p-1} = g_{p-1} with the preconditioner on levels 0..p-1, then the
recovery of u^p. Checked against the oracle's direct solve of the full system
and the oracle's own reduced iteration."""
import numpy as np
import pytest

import sg_inputs as S
from oracle import hsc, sg_operator as so
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


def _rhs(prob, p, random_top):
    F = S.make_rhs(prob, p)
    if random_top:
        F[:, -3:] = S.random_block(prob.n, 3, seed=8)       # nonzero degree-p columns: g and the recovery
    return F


@pytest.mark.parametrize("ne,M,p,random_top", [(16, 3, 3, False), (16, 3, 3, True), (8, 2, 1, True),
                                                (32, 4, 2, False)])
def test_reduced_solve_fp64_matches_direct_solve(lib, ne, M, p, random_top):
    prob, A, G, off = problem(ne, M, p, sigma=0.3)
    h = lib.SGProblem.from_inputs(prob, p)
    F = _rhs(prob, p, random_top)
    ref = so.direct_solve(A, G, F)
    o = lib.solve_opts(lib.prec_opts(precision=lib.SG_F64, inner_tol=1e-10), precond=lib.SG_PREC_HSC, tol=1e-13,
                       maxit=200, schur_reduced=1, schur_inner_tol=1e-13)
    U, st = lib.sg_solve(h, _t(F), o)
    U = _np(U)
    assert np.abs(U - ref).max() <= 1e-10 * np.abs(ref).max()
    assert st.true_rel_res <= 1e-11


def test_reduced_and_full_iterations_agree_with_oracle(lib):
    """Sec. 5: the preconditioned iterations for A_P and S_{P-1} perform
    identically; the GPU's reduced iteration count equals the oracle's."""
    c = S.CONFIGS["cfg1_fp64_16x16_M3_p3"]
    prob, A, G, off = problem(c["ne"], c["M"], c["p"], c["sigma"], c["corr_len"])
    h = lib.SGProblem.from_inputs(prob, c["p"])
    F = S.make_rhs(prob, c["p"])
    prec = lib.prec_opts(precision=lib.SG_F64, inner_tol=1e-12)
    _, st_full = lib.sg_solve(h, _t(F), lib.solve_opts(prec, precond=lib.SG_PREC_HSC, tol=1e-8))
    _, st_red = lib.sg_solve(h, _t(F), lib.solve_opts(prec, precond=lib.SG_PREC_HSC, tol=1e-8, schur_reduced=1,
                                                       schur_inner_tol=1e-13))
    _, info = hsc.schur_reduced_solve(A, G, off, F, tol=1e-8)
    assert st_red.iterations == info["iters"]
    assert abs(st_red.iterations - st_full.iterations) <= 1


@pytest.mark.parametrize("precond", ["hsc", "mean", "bgs"])
def test_reduced_solve_mixed_oracle_residual(lib, precond):
    """Mixed precision preconditioners on the reduced system, stopped at 1e-8:
    the oracle's FP64 residual of the recovered full solution."""
    prob, A, G, off = problem(64, 4, 3, sigma=0.3)
    h = lib.SGProblem.from_inputs(prob, 3)
    F = S.make_rhs(prob, 3)
    kind = {"hsc": lib.SG_PREC_HSC, "mean": lib.SG_PREC_MEAN, "bgs": lib.SG_PREC_BGS}[precond]
    o = lib.solve_opts(lib.prec_opts(precision=lib.SG_F32), precond=kind, tol=1e-9, schur_reduced=1)
    U, st = lib.sg_solve(h, _t(F), o)
    res = oracle_rel_residual(A, G, F, _np(U))
    assert res <= 1.5e-8, res
    assert st.true_rel_res == pytest.approx(res, rel=1e-3)


def test_reduced_solve_rejections(lib):
    prob, A, G, off = problem(8, 2, 2)
    h = lib.SGProblem.from_inputs(prob, 2)
    F = _t(S.make_rhs(prob, 2))
    with pytest.raises(lib.SGError) as e:
        lib.sg_solve(h, F, lib.solve_opts(schur_reduced=1, use_x0=1), U=F.clone())
    assert e.value.status == 1
    h0 = lib.SGProblem(8, 8, 2, 0, prob.rowptr, prob.colidx, prob.vals)
    with pytest.raises(lib.SGError) as e:
        lib.sg_solve(h0, _t(S.make_rhs(prob, 0)), lib.solve_opts(schur_reduced=1))
    assert e.value.status == 1
    b = lib.SGBatch([h])
    with pytest.raises(lib.SGError) as e:
        b.solve([F], lib.solve_opts(schur_reduced=1))
    assert e.value.status == 7
    b.close()
