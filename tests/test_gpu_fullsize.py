"""Parity of the CUDA path with the FP64 oracle at the full sizes of the
measured workloads, in the launch shapes the benchmark times (autotuned SG
products), plus forced shapes that reach the other kernel instantiations:

* 128 x 128 grid, M = 6, p = 4 (P = 210): mixed and all-FP64 HSC solves
  against the oracle's flexible CG with exact Algorithm 1 (element by element),
  and the timed solve (rel.res 1e-8) against the oracle's FP64 residual;
* 512 x 512 grid, M = 10, p = 4 (P = 1001): the SG product (FP64, FP32) and the
  level-p products of the mixed preconditioner on sampled rows, and the timed
  mixed solve against the oracle's FP64 residual;
* the 64 seeded systems of the batched workload solved in one batch, each
  against the oracle's FP64 residual.

The result is the solution of eq. (global-system) (Sec. 2). Tolerances: the
solution error is about kappa(A) times the residual, so the element checks
solve to 1e-12 (mixed) / 1e-13 (FP64) and compare at 1e-7 / 1e-10 of max|u|;
the timed solves stop at 1e-8 and the oracle's FP64 residual must be
<= 1.5e-8; the products keep the rounding bounds of the small-size tests.
"""
import math

import numpy as np
import pytest

import sg_inputs as S
from oracle import chaos, hsc, krylov, sg_operator as so
from tests.gpu_common import TOL32, TOL64, oracle_rel_residual, sample_rows

pytestmark = pytest.mark.gpu

# bench.py's options for the timed solve: mixed HSC, FP64 top level, inner tol 1e-2, rel.res 1e-8
TIMED = dict(inner_tol=1e-2, tol=1e-8)


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


def _timed_opts(L, check=0, df64=0):
    return L.solve_opts(L.prec_opts(precision=L.SG_F32, top_level_f64=1, inner_tol=TIMED["inner_tol"], df64=df64),
                        precond=L.SG_PREC_HSC, tol=TIMED["tol"], maxit=500, check_true_residual=check)


class _Case:
    pass


def _case(lib, name):
    c = S.CONFIGS[name]
    k = _Case()
    k.cfg = c
    k.prob = S.make_problem(c["ne"], c["M"], c["sigma"], c["corr_len"])
    k.A = so.kl_matrices(k.prob.rowptr, k.prob.colidx, k.prob.vals)
    k.G = chaos.g_matrices(c["M"], c["p"])
    _, k.off = chaos.multi_indices(c["M"], c["p"])
    k.F = S.make_rhs(k.prob, c["p"])
    k.h = lib.SGProblem.from_inputs(k.prob, c["p"])
    lib.sg_autotune(k.h)
    k.tuned = lib.sg_autotune_shapes(k.h)
    return k


# --------------------------------------------------------------- 128 x 128

@pytest.fixture(scope="module")
def cfg2(lib):
    k = _case(lib, "cfg2_mixed_128x128_M6_p4")
    a0 = hsc.A0Solver(k.A[0])
    k.ref, info = krylov.fcg(lambda X: so.sg_apply(k.A, k.G, X), k.F,
                             lambda R: hsc.hsc_apply(k.A, k.G, k.off, R, a0solve=a0), tol=1e-13, maxit=100)
    assert info["converged"]
    return k


@pytest.mark.parametrize("df64", [0, 1])
def test_cfg2_mixed_solve_matches_oracle(lib, cfg2, df64):
    """Mixed precision (FP32 inner solves and level products, FP64 outer CG and
    top level; df64: the outer product and the level-p products in
    double-float arithmetic) solved to 1e-12: within 1e-7 of the oracle's
    solution."""
    o = lib.solve_opts(lib.prec_opts(precision=lib.SG_F32, top_level_f64=1, inner_tol=1e-2, df64=df64),
                       precond=lib.SG_PREC_HSC, tol=1e-12, maxit=200)
    U, st = lib.sg_solve(cfg2.h, _t(cfg2.F), o)
    U = _np(U)
    scale = np.abs(cfg2.ref).max()
    assert np.abs(U - cfg2.ref).max() <= 1e-7 * scale, np.abs(U - cfg2.ref).max() / scale
    # attainable true residual: the outer product's rounding relative to the
    # stencil's cancellation (sum |terms| / |result| ~ 1/h^2 = 1.6e4 here) times
    # 2^-53 (FP64) or 2^-47 (double-float)
    assert oracle_rel_residual(cfg2.A, cfg2.G, cfg2.F, U) <= (1.5e-12 if not df64 else 2e-11)


def test_cfg2_fp64_solve_matches_oracle(lib, cfg2):
    """All FP64 solved to 1e-13: within 1e-10 of the oracle's solution."""
    o = lib.solve_opts(lib.prec_opts(precision=lib.SG_F64, inner_tol=1e-2), precond=lib.SG_PREC_HSC, tol=1e-13,
                       maxit=200)
    U, st = lib.sg_solve(cfg2.h, _t(cfg2.F), o)
    U = _np(U)
    scale = np.abs(cfg2.ref).max()
    assert np.abs(U - cfg2.ref).max() <= 1e-10 * scale, np.abs(U - cfg2.ref).max() / scale


@pytest.mark.parametrize("df64", [0, 1])
def test_cfg2_timed_solve_oracle_residual(lib, cfg2, df64):
    """The benchmark's solve (rel.res 1e-8): the oracle's FP64 residual of the
    GPU solution, and the iteration count the CPU baseline is scaled by."""
    import bench
    U, st = lib.sg_solve(cfg2.h, _t(cfg2.F), _timed_opts(lib, check=1, df64=df64))
    res = oracle_rel_residual(cfg2.A, cfg2.G, cfg2.F, _np(U))
    assert res <= 1.5e-8, res
    assert st.true_rel_res == pytest.approx(res, rel=1e-3)
    assert st.iterations == bench.WORKLOADS["cfg2"]["hsc_iterations"]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_cfg2_sg_apply_autotuned_parity(lib, cfg2, prec):
    import torch
    from tests.gpu_common import abs_bound
    U = S.random_block(cfg2.prob.n, cfg2.h.P, seed=1205)
    dt = torch.float64 if prec == "f64" else torch.float32
    if prec == "f32":
        U = U.astype(np.float32).astype(np.float64)
    Y = _np(lib.sg_apply(cfg2.h, _t(U, dt)))
    ref = so.sg_apply(cfg2.A, cfg2.G, U)
    tol = TOL64 if prec == "f64" else TOL32
    assert np.all(np.abs(Y - ref) <= tol * abs_bound(cfg2.A, cfg2.G, U) + 1e-300)


# --------------------------------------------------------------- 512 x 512

@pytest.fixture(scope="module")
def cfg5(lib):
    return _case(lib, "cfg5_large_512x512_M10_p4")


# (threads, pair form) pins beside the autotuned shapes: at P = 1001 these are
# 1 output per thread on 1024 threads, 2 on 512, 4 on 256 and 8 on 128
SHAPES = [None, (1024, 1), (512, 0), (512, 1), (256, 1), (128, 0)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "tuned" if s is None else f"t{s[0]}_pair{s[1]}")
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_cfg5_sg_apply_sampled_rows(lib, cfg5, shape, prec):
    """The full SG product at P = 1001 against the oracle on sampled rows."""
    import torch
    h = cfg5.h
    if shape is not None:
        t, pr = shape
        lib.sg_autotune_set(h, t, t, cfg5.tuned[2], pr, pr, cfg5.tuned[5])
    try:
        U = S.random_block(cfg5.prob.n, h.P, seed=1205)
        dt = torch.float64 if prec == "f64" else torch.float32
        if prec == "f32":
            U = U.astype(np.float32)
        Ud = _t(U, dt)
        Y = lib.sg_apply(h, Ud)
        rows = sample_rows(cfg5.prob.n, seed=5)
        Yr = _np(Y[torch.as_tensor(rows, device="cuda")])
        del Y, Ud
        U = U.astype(np.float64)
        ref = so.sg_apply_rows(cfg5.A, cfg5.G, U, rows)
        bound = so.sg_apply_rows([abs(a) for a in cfg5.A], [abs(g) for g in cfg5.G], np.abs(U), rows)
        tol = TOL64 if prec == "f64" else TOL32
        assert np.all(np.abs(Yr - ref) <= tol * bound + 1e-300), np.max(np.abs(Yr - ref) / (bound + 1e-300))
    finally:
        lib.sg_autotune_set(h, *cfg5.tuned)


@pytest.mark.parametrize("df64", [0, 1])
@pytest.mark.parametrize("lvl", ["pre", "post"])
def test_cfg5_top_level_products_sampled_rows(lib, cfg5, lvl, df64):
    """The level-p products of the mixed preconditioner (FP32 input, FP64 or
    double-float accumulation, FP64 residual, FP32 output): B_p (715 -> 220
    columns) and C_p (220 -> 715) at M = 10, p = 4, on sampled rows."""
    import torch
    p, off = cfg5.cfg["p"], cfg5.off
    lo, li = (p - 1, p) if lvl == "pre" else (p, p - 1)
    win, wout = off[li + 1] - off[li], off[lo + 1] - off[lo]
    X = S.random_block(cfg5.prob.n, win, seed=31).astype(np.float32)
    Yin = S.random_block(cfg5.prob.n, wout, seed=32)
    Y = lib.sg_level_apply(cfg5.h, lo, li, _t(X, torch.float32), _t(Yin), df64=bool(df64))
    assert Y.dtype == torch.float32
    rows = sample_rows(cfg5.prob.n, seed=6)
    Yr = _np(Y[torch.as_tensor(rows, device="cuda")])
    X = X.astype(np.float64)
    exact = Yin[rows] - so.level_apply(cfg5.A, cfg5.G, off, lo, li, X, rows=rows)
    bound = np.abs(Yin[rows]) + so.level_apply([abs(a) for a in cfg5.A], [abs(g) for g in cfg5.G], off, lo, li,
                                               np.abs(X), rows=rows)
    # FP64 (or double-float: m 2^-46 per sum of m <= 99 products here) arithmetic,
    # then one rounding of the result to FP32
    err = np.abs(Yr - exact)
    tol = TOL64 if not df64 else 99 * 2.0 ** -46
    assert np.all(err <= tol * bound + 6e-8 * np.abs(exact) + 1e-300)


@pytest.mark.parametrize("outer", ["tuned", "t512_pair1", "tuned_df64", "t512_pair1_df64"])
def test_cfg5_timed_solve_oracle_residual(lib, cfg5, outer):
    """The benchmark's mixed solve at 512 x 512, M = 10, p = 4 (261M unknowns)
    stopped at 1e-8: the oracle's FP64 residual of the GPU solution. The
    t512 cases pin the fused outer product to 512 threads in pair form (two
    outputs per thread); the df64 cases run the outer product and the level-p
    products in double-float arithmetic (the benchmark's headline solve)."""
    import bench
    h = cfg5.h
    df64 = 1 if outer.endswith("df64") else 0
    if outer.startswith("t512"):
        t = cfg5.tuned
        lib.sg_autotune_set(h, t[0], t[1], 512, t[3], t[4], 1)
    try:
        U, st = lib.sg_solve(h, _t(cfg5.F), _timed_opts(lib, check=1, df64=df64))
        res = oracle_rel_residual(cfg5.A, cfg5.G, cfg5.F, _np(U))
        del U
    finally:
        lib.sg_autotune_set(h, *cfg5.tuned)
    assert res <= 1.5e-8, res
    assert st.true_rel_res == pytest.approx(res, rel=1e-3)
    if outer in ("tuned", "tuned_df64"):
        assert st.iterations == bench.WORKLOADS["cfg5"]["hsc_iterations"]


# ------------------------------------------------------------------ batch

def test_cfg3_batch_each_system_oracle_residual(lib):
    """The 64 seeded systems of the batched workload (meshes 32^2..256^2, M 2..8,
    p 2..4), autotuned and solved in one batch with the benchmark's options:
    the oracle's FP64 residual of every system's solution."""
    from concurrent.futures import ThreadPoolExecutor
    cfgs = S.draw_batch_configs(64, seed=1864)
    probs, hs, Fs = [], [], []
    for c in cfgs:
        prob = S.make_problem(c["ne"], c["M"], c["sigma"], c["corr_len"])
        h = lib.SGProblem.from_inputs(prob, c["p"])
        lib.sg_autotune(h)
        probs.append(prob)
        hs.append(h)
        Fs.append(S.make_rhs(prob, c["p"]))
    batch = lib.SGBatch(hs)
    Us, st = batch.solve([_t(F) for F in Fs], _timed_opts(lib, check=1))
    Us = [_np(U) for U in Us]
    batch.close()

    def residual(i):
        c, prob = cfgs[i], probs[i]
        A = so.kl_matrices(prob.rowptr, prob.colidx, prob.vals)
        G = chaos.g_matrices(c["M"], c["p"])
        return float(np.linalg.norm(Fs[i] - so.sg_apply(A, G, Us[i])) / np.linalg.norm(Fs[i]))

    with ThreadPoolExecutor(16) as ex:
        res = list(ex.map(residual, range(len(cfgs))))
    assert all(s.status == 0 for s in st)
    assert max(res) <= 1.5e-8, max(res)
    for s, r in zip(st, res):
        assert s.true_rel_res == pytest.approx(r, rel=1e-3, abs=1e-12)
    assert [h.P for h in hs] == [math.comb(c["M"] + c["p"], c["M"]) for c in cfgs]
