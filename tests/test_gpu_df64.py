"""Double-float arithmetic (FP32 pairs on the FP32 units) in the products
that read the mixed preconditioner's FP32 output: the level-p products and
the outer solve's SG product, against the oracle and against their FP64
counterparts."""
import numpy as np
import pytest

import sg_inputs as S
from oracle import sg_operator as so
from tests.gpu_common import oracle_rel_residual, problem

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


@pytest.mark.parametrize("ne,M,p", [(16, 3, 3), (8, 6, 4), (32, 10, 2)])
def test_df64_level_products_against_oracle(lib, ne, M, p):
    """Every level product B_l, C_l with FP32 input and double-float
    accumulation: within m 2^-46 sum|terms| (m products per entry) plus one
    FP32 rounding of the result of the exact value, with values spanning
    several orders of magnitude (scaled columns)."""
    import torch
    prob, A, G, off = problem(ne, M, p)
    h = lib.SGProblem.from_inputs(prob, p)
    rng = np.random.default_rng(7)
    m = 9 * (1 + 2 * M)
    for lo, li in [(l - 1, l) for l in range(1, p + 1)] + [(l, l - 1) for l in range(1, p + 1)]:
        win, wout = off[li + 1] - off[li], off[lo + 1] - off[lo]
        X = (S.random_block(prob.n, win, seed=lo + 10 * li) * 10.0 ** rng.integers(-3, 4, size=win)).astype(np.float32)
        Yin = S.random_block(prob.n, wout, seed=5 + lo)
        Y = _np(lib.sg_level_apply(h, lo, li, _t(X, torch.float32), _t(Yin), df64=True))
        Y64 = _np(lib.sg_level_apply(h, lo, li, _t(X, torch.float32), _t(Yin), df64=False))
        X = X.astype(np.float64)
        exact = Yin - so.level_apply(A, G, off, lo, li, X)
        bound = np.abs(Yin) + so.level_apply([abs(a) for a in A], [abs(g) for g in G], off, lo, li, np.abs(X))
        assert np.all(np.abs(Y - exact) <= m * 2.0 ** -46 * bound + 6e-8 * np.abs(exact) + 1e-300), (lo, li)
        # the FP64-accumulating product rounds to the same FP32 value almost everywhere
        assert np.mean(Y == Y64) > 0.99


@pytest.mark.parametrize("ne,M,p,gpc,generic", [(16, 3, 3, False, False), (8, 10, 4, False, False),
                                                (7, 6, 6, False, False), (8, 10, 4, False, True),
                                                (8, 3, 2, True, False)])
def test_df64_full_product_against_oracle(lib, ne, M, p, gpc, generic, monkeypatch):
    """Y = sum_k A_k U G_k^T with FP32 U, double-float sums, FP64 Y: within
    m 2^-46 sum|terms| (m the products of an entry) of the exact product, on
    the staged pair kernel (P = 84, 1001, 924, and the gPC coefficient's
    dense coupling) and on the row-per-warp kernel (staged kernels off)."""
    import torch
    if generic:
        monkeypatch.setenv("SGHSC_GENERIC_PRODUCTS", "1")
    if gpc:
        from tests.test_gpu_lognormal import _case
        prob, A, G, off = _case(ne, M, p)
    else:
        prob, A, G, off = problem(ne, M, p)
    h = lib.SGProblem.from_inputs(prob, p)
    rng = np.random.default_rng(3)
    U = (S.random_block(prob.n, h.P, seed=4) * 10.0 ** rng.integers(-3, 4, size=h.P)).astype(np.float32)
    Y = _np(lib.sg_apply(h, _t(U, torch.float32), df64=True))
    U = U.astype(np.float64)
    exact = so.sg_apply(A, G, U)
    bound = so.sg_apply([abs(a) for a in A], [abs(g) for g in G], np.abs(U))
    per_out = max(int(sum((g != 0).sum(axis=1).max() for g in G)), 1)
    m = 9 * (per_out + 1)
    assert np.all(np.abs(Y - exact) <= m * 2.0 ** -46 * bound + 2.0 ** -52 * np.abs(exact) + 1e-300)
    with pytest.raises(ValueError):
        lib.sg_apply(h, _t(U), df64=True)
    h.close()


@pytest.mark.parametrize("precond", ["hsc", "bgs"])
def test_df64_mixed_solve_matches_oracle(lib, precond):
    """Mixed solves with the double-float outer and top-level products to
    1e-12: within 1e-7 of the oracle's direct solve, like the FP64 products."""
    c = S.CONFIGS["cfg1_fp64_16x16_M3_p3"]
    prob, A, G, off = problem(c["ne"], c["M"], c["p"], c["sigma"], c["corr_len"])
    h = lib.SGProblem.from_inputs(prob, c["p"])
    F = S.make_rhs(prob, c["p"])
    ref = so.direct_solve(A, G, F)
    kind = lib.SG_PREC_HSC if precond == "hsc" else lib.SG_PREC_BGS
    o = lib.solve_opts(lib.prec_opts(precision=lib.SG_F32, df64=1), precond=kind, tol=1e-12)
    U, st = lib.sg_solve(h, _t(F), o)
    assert np.abs(_np(U) - ref).max() <= 1e-7 * np.abs(ref).max()
    assert st.true_rel_res <= 2e-12


def test_df64_and_fp64_outer_products_take_the_same_iterations(lib):
    """At the benchmark's tolerance the two arithmetics of the outer product
    give the same iteration count and residuals agreeing to FP64-class
    accuracy; the oracle's residual of the double-float solution meets 1e-8."""
    prob, A, G, off = problem(64, 6, 3, sigma=0.3, corr=1.0)
    h = lib.SGProblem.from_inputs(prob, 3)
    lib.sg_autotune(h)
    F = S.make_rhs(prob, 3)
    out = {}
    for df in (0, 1):
        o = lib.solve_opts(lib.prec_opts(precision=lib.SG_F32, df64=df), precond=lib.SG_PREC_HSC, tol=1e-8)
        U, st = lib.sg_solve(h, _t(F), o)
        out[df] = (st, _np(U))
    assert out[0][0].iterations == out[1][0].iterations
    # the FP32 preconditioner amplifies the last-bit differences of the two
    # arithmetics from one iteration to the next: histories agree to 1e-3
    for a, b in zip(out[0][0].res_hist, out[1][0].res_hist):
        assert a == pytest.approx(b, rel=1e-3)
    assert oracle_rel_residual(A, G, F, out[1][1]) <= 1.5e-8
