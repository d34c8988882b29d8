"""The gPC (lognormal) coefficient of Sec. 6 on the GPU: the block-dense SG
product against the oracle, Algorithm 1 with non-block-diagonal D_l (nested
level CG) against the oracle's exact Algorithm 1, whole solves against the
oracle's iteration counts and condition estimates, and the paper's Tables 6-9
(soft, as the oracle's pins)."""
import math
import os

import numpy as np
import pytest

import sg_inputs as S
from oracle import chaos, hsc, krylov, sg_operator as so
from tests.gpu_common import oracle_rel_residual

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


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


def _case(ne, M, p, cov=1.0):
    prob = S.make_lognormal_problem(ne, M, cov, 0.5, 2 * p)
    A = so.kl_matrices(prob.rowptr, prob.colidx, prob.vals)
    G = chaos.gpc_g_matrices(M, p, 2 * p)
    _, off = chaos.multi_indices(M, p)
    return prob, A, G, off


def _tight(L, kind, **kw):
    o = L.prec_opts(precision=L.SG_F64, inner_tol=1e-12, level_tol=1e-12, level_maxit=2000, **kw)
    return L.solve_opts(o, precond=kind, tol=1e-8, maxit=1000)


@pytest.mark.parametrize("ne,M,p", [(8, 2, 2), (16, 3, 2), (8, 4, 3)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_gpc_sg_apply_parity(lib, ne, M, p, prec):
    """Y = sum_i A_i U G_i^T with every coefficient term up to degree 2p; the
    rounding bound is m u sum|terms| with m the largest number of products
    summed into one entry (9 nonzeros times the couplings of an output)."""
    import torch
    prob, A, G, off = _case(ne, M, p)
    h = lib.SGProblem.from_inputs(prob, p)
    assert h.q == 2 * p and h.nterm == math.comb(M + 2 * p, M)
    U = S.random_block(prob.n, h.P, seed=3)
    dt = torch.float64 if prec == "f64" else torch.float32
    if prec == "f32":
        U = U.astype(np.float32).astype(np.float64)
    Y = _np(lib.sg_apply(h, _t(U, dt)))
    ref = so.sg_apply(A, G, U)
    bound = so.sg_apply([abs(a) for a in A], [abs(g) for g in G], np.abs(U))
    per_out = max(int(sum((g != 0).sum(axis=1).max() for g in G)), 1)
    m = 9 * (per_out + 1)
    u = 1.2e-16 if prec == "f64" else 6.0e-8
    assert np.all(np.abs(Y - ref) <= m * u * bound + 1e-300)


def test_gpc_hsc_matches_exact_algorithm1(lib):
    """Algorithm 1 with B_l / C_l reaching every lower degree and the nested
    level CG for D_l (tolerances 1e-12) against the oracle's Algorithm 1 with
    exact factorisations of D_l."""
    prob, A, G, off = _case(8, 3, 3)
    h = lib.SGProblem.from_inputs(prob, 3)
    R = S.random_block(prob.n, h.P, seed=5)
    o = lib.prec_opts(precision=lib.SG_F64, inner_tol=1e-13, level_tol=1e-13, level_maxit=2000)
    Z = _np(lib.hsc_precond_apply(h, _t(R), o))
    ref = hsc.hsc_apply(A, G, off, R, general=True)
    assert np.abs(Z - ref).max() <= 1e-9 * np.abs(ref).max()


def test_gpc_mean_preconditioner_and_unsupported_paths(lib):
    prob, A, G, off = _case(8, 2, 2)
    h = lib.SGProblem.from_inputs(prob, 2)
    R = S.random_block(prob.n, h.P, seed=6)
    Z = _np(lib.mean_precond_apply(h, _t(R), lib.prec_opts(precision=lib.SG_F64, inner_tol=1e-13)))
    assert np.abs(Z - hsc.mean_apply(A, R)).max() <= 1e-10 * np.abs(Z).max()
    for call, o in ((lib.bgs_precond_apply, lib.prec_opts(precision=lib.SG_F64)),
                    (lib.hsc_precond_apply, lib.prec_opts(precision=lib.SG_F32))):
        with pytest.raises(lib.SGError) as e:
            call(h, _t(R), o)
        assert e.value.status == 7
    with pytest.raises(lib.SGError):
        lib.SGProblem(8, 8, 2, 2, prob.rowptr, prob.colidx, prob.vals, family=lib.SG_LEGENDRE, q=4)


@pytest.mark.parametrize("M,p", [(1, 4), (2, 4), (4, 1), (4, 2)])
def test_gpc_solves_match_oracle(lib, M, p):
    """Whole solves at the paper's lognormal setting (10x10 mesh, CoV 100 %):
    with tight nested tolerances the GPU takes the oracle's iteration counts
    (exact inner solves) and its condition estimates to 1e-3, and the
    oracle's FP64 residual of the GPU solution is below 1.5e-8."""
    from tests.test_oracle_krylov import _lognormal_run
    prob, A, G, off = _case(10, M, p)
    h = lib.SGProblem.from_inputs(prob, p)
    F = S.make_rhs(prob, p)
    ref = _lognormal_run(M, p, 1.0)
    for name, kind in (("mean", lib.SG_PREC_MEAN), ("hsc", lib.SG_PREC_HSC)):
        U, st = lib.sg_solve(h, _t(F), _tight(lib, kind, m0=lib.SG_M0_DIAG))
        assert st.iterations == ref[name][0], name
        assert st.kappa_est == pytest.approx(ref[name][1], rel=1e-3), name
        assert oracle_rel_residual(A, G, F, _np(U)) <= 1.5e-8


def _read(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


def _gpu_row(lib, ne, M, p, cov):
    prob = S.make_lognormal_problem(ne, M, cov, 0.5, 2 * p)
    h = lib.SGProblem.from_inputs(prob, p)
    F = _t(S.make_rhs(prob, p))
    out = {}
    for name, kind in (("mean", lib.SG_PREC_MEAN), ("hsc", lib.SG_PREC_HSC)):
        o = lib.solve_opts(lib.prec_opts(precision=lib.SG_F64, m0=lib.SG_M0_DIAG, inner_tol=1e-8, level_tol=1e-8,
                                         level_maxit=2000, inner_maxit=1000), precond=kind, tol=1e-8, maxit=1000)
        _, st = lib.sg_solve(h, F, o)
        out[name] = (st.iterations, st.kappa_est)
    h.close()
    return out


def _soft(out, m_it, m_k, h_it, h_k):
    for (it, k), (pit, pk) in ((out["mean"], (m_it, m_k)), (out["hsc"], (h_it, h_k))):
        assert abs(it - pit) <= max(3, 0.25 * pit)
        assert k == pytest.approx(pk, rel=0.25)
    assert out["hsc"][1] < out["mean"][1] and 2 * out["hsc"][0] < out["mean"][0] + 2


@pytest.mark.parametrize("row", _read("sec6_table6_lognormal_vary_N.txt"), ids=lambda r: f"N{int(r[0])}")
def test_paper_table6_lognormal_on_gpu(lib, row):
    N, _, _, _, m_it, m_k, _, _, h_it, h_k = row
    _soft(_gpu_row(lib, 10, int(N), 4, 1.0), m_it, m_k, h_it, h_k)


@pytest.mark.parametrize("row", _read("sec6_table7_lognormal_vary_P.txt"), ids=lambda r: f"P{int(r[0])}")
def test_paper_table7_lognormal_on_gpu(lib, row):
    p, _, _, _, m_it, m_k, _, _, h_it, h_k = row
    _soft(_gpu_row(lib, 10, 4, int(p), 1.0), m_it, m_k, h_it, h_k)


@pytest.mark.parametrize("row", [r for r in _read("sec6_table8_lognormal_vary_cov.txt") if r[0] <= 100],
                         ids=lambda r: f"cov{int(r[0])}")
def test_paper_table8_lognormal_on_gpu(lib, row):
    cov, _, _, m_it, m_k, _, _, h_it, h_k = row
    _soft(_gpu_row(lib, 10, 4, 4, cov / 100.0), m_it, m_k, h_it, h_k)


@pytest.mark.parametrize("row", [r for r in _read("sec6_table9_lognormal_vary_h.txt") if r[0] <= 20],
                         ids=lambda r: f"h1_{int(r[0])}")
def test_paper_table9_lognormal_on_gpu(lib, row):
    inv_h, _, _, _, m_it, m_k, _, _, h_it, h_k = row
    _soft(_gpu_row(lib, int(inv_h), 4, 4, 1.0), m_it, m_k, h_it, h_k)
