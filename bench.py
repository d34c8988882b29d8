"""Benchmark: time-to-solve of the stochastic Galerkin system at relative
residual 1e-8 with the hierarchical Schur complement preconditioner
(mixed precision: FP32 inner loops, FP64 outer), against the all-FP64
mean-based preconditioner on the same GPU, plus the SG matvec roofline.

Workload (default): 512 x 512 Q1 grid (261121 interior dofs), M = 10 Legendre
variables, p = 4 (P = 1001, 261M unknowns, 2.09 GB per FP64 vector),
sigma = 0.25, correlation length 0.5, f = 1; inner A_0 PCG with a multigrid
V-cycle to 1e-2. ``--workload cfg2`` runs the 128 x 128, M = 6, p = 4 system,
``cfg3`` the 64-system batch.

One step = one full sg_solve (K1 SG matvec, K2 level products, K3/K4 batched
inner PCG + V-cycle, K5 outer FCG) with F resident in HBM. L2 is flushed
(256 MiB write) between timed steps, outside the timed events. The same line
carries the three comparator solves (mean-based FP64, HSC FP64, mean-based
mixed), the SG product alone in FP64 and FP32 against the measured FP64/FP32
ALU rates and the HBM peak, and the end-to-end time from host buffers.

``--impl reference`` times the FP64 CPU oracle (test infrastructure) on a
bounded sample of the same workload on all host cores; that arm is the
deliberately slow baseline, not a target.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import sg_inputs as S  # noqa: E402

METRIC = "time-to-solve at rel.res 1e-8, HSC-PCG vs mean-based PCG; SG matvec HBM GB/s"
# hsc_iterations: outer HSC-FCG iterations of the timed solve (mixed, inner tol
# 1e-2, rel.res 1e-8) as the GPU takes them; the oracle's time per iteration is
# scaled by it in the reference arm, which runs without a GPU (checked by the
# GPU parity tests against the library's own count).
WORKLOADS = {
    "cfg2": dict(name="cfg2_mixed_128x128_M6_p4", hsc_iterations=8, **S.CONFIGS["cfg2_mixed_128x128_M6_p4"]),
    "cfg1": dict(name="cfg1_fp64_16x16_M3_p3", hsc_iterations=6, **S.CONFIGS["cfg1_fp64_16x16_M3_p3"]),
    "cfg4": dict(name="cfg4_64x64_M4_p3", hsc_iterations=6, grad=True, **S.CONFIGS["cfg4_grad_64x64_M4_p3"]),
    "cfg5": dict(name="cfg5_large_512x512_M10_p4", hsc_iterations=7, **S.CONFIGS["cfg5_large_512x512_M10_p4"]),
    # 64 independent systems (mesh, M, p, sigma, L drawn per system), one graph launch
    "cfg3": dict(name="cfg3_batch64_mixed", batch=True, count=64, seed=1864),
}
L2_FLUSH_BYTES = 256 << 20


L2_NOTE = "flushed between timed steps (256 MiB write, outside the events)"


def workload_config(cfg, world):
    """The config object of a workload's line, the same for both arms."""
    if cfg.get("batch"):
        return {"workload": cfg["name"], "systems": cfg["count"], "draw_seed": cfg["seed"], "tol": 1e-8,
                "inner_tol": 1e-2, "l2": L2_NOTE,
                "parallelism": f"systems split over {world} ranks" if world > 1 else "single GPU"}
    P = math.comb(cfg["M"] + cfg["p"], cfg["p"])
    n = (cfg["ne"] - 1) ** 2
    return {"workload": cfg["name"], "ne": cfg["ne"], "M": cfg["M"], "p": cfg["p"], "P": P, "n": n,
            "unknowns": n * P, "sigma": cfg["sigma"], "corr_len": cfg["corr_len"], "inner_tol": 1e-2, "tol": 1e-8,
            "l2": L2_NOTE, "parallelism": "replicas" if world > 1 else "single GPU"}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# DRAM bytes of one FP64 SG-product launch on the 128x128, M=6, p=4 workload:
# dram__bytes_read.sum + dram__bytes_write.sum of an ncu capture of that launch
# (L2 flushed before it, as before each timed launch here).
K1_TRAFFIC = {"cfg2": 35833856 + 119040}
# DRAM bytes of one double-float SG-product launch (sg_apply SG_F32_ACCDF64):
# dram__bytes_read.sum + dram__bytes_write.sum of an ncu capture of the current
# kernel on the 255^2 grid of the same operator (447176192 + 475274752 bytes,
# L2 flushed before the launch), scaled by the rows to the 511^2 grid
# (x 261121 / 65025; the traffic is per row: the row's values, its neighbour
# rows of U from L2, its row of Y).
DF_TRAFFIC = {"cfg5": int((447176192 + 475274752) * 261121 / 65025)}
# FP32 operations of one double-float multiply-add a * x + s (a double-float,
# x FP32): the exact product (FMUL, FFMA for its error, FFMA for a.lo x) and
# the two-sum accumulation (six FADD for the hi parts and their error, two
# for the lo parts). The double-float peak is the measured FP32 FMA-chain rate
# (two flops per FMA) divided by this count.
DF_OPS_PER_MAC = 11


class ClockSampler:
    """nvidia-smi samples (every 50 ms) during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def sg_matvec_bytes(n, nnz, M, P, es):
    """Algorithmic bytes of one SG product: pattern once, M+1 values per
    nonzero, U read once, Y written once."""
    return 4 * (n + 1) + 4 * nnz + es * (M + 1) * nnz + 2 * es * n * P


def sg_matvec_bytes_df(n, nnz, M, P):
    """Algorithmic bytes of the double-float product: pattern once, M+1
    double-float values (8 bytes) per nonzero, FP32 U read once, FP64 Y
    written once."""
    return 4 * (n + 1) + 4 * nnz + 8 * (M + 1) * nnz + 4 * n * P + 8 * n * P


def _comb(a, b):
    return math.comb(a, b) if 0 <= b <= a else 0


def sg_pairs(M, p):
    """Distinct (k, j) among the couplings alpha_j = alpha_l +- e_k: per k, the
    j of degree < p (a neighbour j + e_k) and the j of degree p with j_k >= 1."""
    if p < 1 or M < 1:
        return 0
    return M * (_comb(M + p - 1, M) + _comb(M + p - 1, M - 1) - _comb(M + p - 2, M - 2))


def sg_matvec_flops(n, nnz, M, p, P, n_m):
    """Multiply-adds of the least-work form of the full product: per nonzero P
    (G_0 = I) + one per distinct (k, j) pair, per row one per off-diagonal G
    entry (the coupling weights)."""
    return 2 * nnz * (P + sg_pairs(M, p)) + 2 * n * n_m


def build_problem(cfg):
    prob = S.make_problem(cfg["ne"], cfg["M"], cfg["sigma"], cfg["corr_len"])
    return prob


def run_ours(args, rank, world, dev):
    import torch

    import paper_1205_1864_gb300 as L
    cfg = WORKLOADS[args.workload]
    t0 = time.time()
    prob = build_problem(cfg)
    p = cfg["p"]
    h = L.SGProblem.from_inputs(prob, p)
    tuned = L.sg_autotune(h)   # block sizes of the SG product (FP64, FP32), part of setup
    forms = L.sg_autotune_forms(h)   # pair (1) or gather (0) form: FP64, FP32, outer
    # inner solver per degree-level width: 0 stand-alone kernels, 1 / 3 on-chip
    # cluster solver with 8 / 16 CTAs, 2 the wide one
    _, _off = h.chaos_table()
    inner_paths = {int(_off[l + 1] - _off[l]): h.inner_path(int(_off[l + 1] - _off[l])) for l in range(p + 1)}
    setup_s = time.time() - t0
    n, P, M, nnz = h.n, h.P, h.M, h.nnz
    alpha, off = h.chaos_table()
    n_m = int(2 * M * math.comb(M + p - 1, M))
    F_np = S.make_rhs(prob, p)
    F = torch.tensor(F_np, dtype=torch.float64, device=dev)
    U = torch.empty_like(F)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    # headline: mixed HSC, the products that read the FP32 preconditioner output in double-float arithmetic
    hsc_opts = L.solve_opts(L.prec_opts(precision=L.SG_F32, top_level_f64=1, inner_tol=1e-2, df64=1),
                            precond=L.SG_PREC_HSC, tol=1e-8, maxit=500, check_true_residual=0)
    hsc_f64prod_opts = L.solve_opts(L.prec_opts(precision=L.SG_F32, top_level_f64=1, inner_tol=1e-2, df64=0),
                                    precond=L.SG_PREC_HSC, tol=1e-8, maxit=500, check_true_residual=0)
    mean_opts = L.solve_opts(L.prec_opts(precision=L.SG_F64, inner_tol=1e-2), precond=L.SG_PREC_MEAN,
                             tol=1e-8, maxit=500, check_true_residual=0)
    hsc64_opts = L.solve_opts(L.prec_opts(precision=L.SG_F64, inner_tol=1e-2), precond=L.SG_PREC_HSC,
                              tol=1e-8, maxit=500, check_true_residual=0)
    mean32_opts = L.solve_opts(L.prec_opts(precision=L.SG_F32, inner_tol=1e-2, df64=1), precond=L.SG_PREC_MEAN,
                               tol=1e-8, maxit=500, check_true_residual=0)

    def timed_solves(opts, steps, warmup, count_launches=False):
        for _ in range(warmup):
            L.sg_solve(h, F, opts, U)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ts, stats = [], None
        l0 = L._lib.LIB.sg_kernel_launches()
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, stats = L.sg_solve(h, F, opts, U)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        launches = L._lib.LIB.sg_kernel_launches() - l0
        return ts, stats, launches

    if args.profile == "apply":
        # the SG product alone, FP64, FP32, then FP32 in / double-float sums /
        # FP64 out (warm-up + timed launches each)
        out = {"profile": "apply", "workload": cfg["name"], "n": n, "P": P, "nnz": nnz}
        for name, dt, es, df in (("fp64", torch.float64, 8, False), ("fp32", torch.float32, 4, False),
                                 ("df64", torch.float32, 0, True)):
            Ut = torch.tensor(S.random_block(n, P, seed=1205), dtype=dt, device=dev)
            Yt = torch.empty(Ut.shape, dtype=torch.float64 if df else dt, device=dev)
            for _ in range(args.warmup):
                L.sg_apply(h, Ut, Yt, df64=df)
            ts = []
            for _ in range(args.steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                L.sg_apply(h, Ut, Yt, df64=df)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            k = float(np.mean(ts))
            b = sg_matvec_bytes_df(n, nnz, M, P) if df else sg_matvec_bytes(n, nnz, M, P, es)
            fl = sg_matvec_flops(n, nnz, M, p, P, n_m)
            out[name] = {"ms": k, "GB_s": b / k / 1e6, "TFLOP_s": fl / k / 1e9, "bytes": b, "flops": fl}
            del Ut, Yt
        return out
    if args.profile == "levels":
        # every level product B_l, C_l alone: FP32, FP64, FP32 in with FP64
        # sums and with double-float sums (warm-up + timed launches each)
        alpha, off = h.chaos_table()
        out = {"profile": "levels", "workload": cfg["name"], "n": n, "nnz": nnz, "products": []}
        for lo, li in [(l - 1, l) for l in range(1, p + 1)] + [(l, l - 1) for l in range(1, p + 1)]:
            win, wout = int(off[li + 1] - off[li]), int(off[lo + 1] - off[lo])
            ai, ao = alpha[off[li]:off[li + 1]], alpha[off[lo]:off[lo + 1]]
            couplings = sum(int((np.abs(ao - a).sum(axis=1) == 1).sum()) for a in ai)   # alpha_out = alpha_in +- e_k
            rec = {"out": lo, "in": li, "w_out": wout, "w_in": win, "couplings": couplings,
                   "gather_flops": 2 * nnz * couplings}
            for name, tx, ty, df in (("fp32", torch.float32, torch.float32, False),
                                     ("fp64", torch.float64, torch.float64, False),
                                     ("fp32_acc64", torch.float32, torch.float64, False),
                                     ("fp32_accdf64", torch.float32, torch.float64, True)):
                X = torch.tensor(S.random_block(n, win, seed=lo + 10 * li), dtype=tx, device=dev)
                Yin = torch.tensor(S.random_block(n, wout, seed=5 + lo), dtype=ty, device=dev)
                Yo = torch.empty((n, wout), dtype=tx, device=dev)
                for _ in range(args.warmup):
                    L.sg_level_apply(h, lo, li, X, Yin, Yo, df64=df)
                ts = []
                for _ in range(args.steps):
                    flush.zero_()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    L.sg_level_apply(h, lo, li, X, Yin, Yo, df64=df)
                    e1.record(stream)
                    e1.synchronize()
                    ts.append(e0.elapsed_time(e1))
                rec[name + "_ms"] = float(np.mean(ts))
                del X, Yin, Yo
            out["products"].append(rec)
        return out
    if args.profile == "inner":
        # the batched inner PCG on A_0 alone, FP32, one batch as wide as the widest degree level
        wmax = max(int(math.comb(M + l - 1, l)) for l in range(1, p + 1))
        B = torch.tensor(S.random_block(n, wmax, seed=1205), dtype=torch.float32, device=dev)
        po = L.prec_opts(precision=L.SG_F32, inner_tol=1e-2)
        for _ in range(args.warmup):
            L.sg_inner_solve(h, B, po)
        ts = []
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, its = L.sg_inner_solve(h, B, po)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return {"profile": "inner", "workload": cfg["name"], "w": wmax, "ms": float(np.mean(ts)),
                "iterations": int(its.max())}
    if args.profile:
        ts, st_h, launches = timed_solves(hsc_opts, args.steps, args.warmup)
        return {"profile": "solve", "workload": cfg["name"], "ms": float(np.mean(ts)), "iterations": st_h.iterations,
                "launches_per_solve": int(launches / max(args.steps, 1)), "autotuned_threads_f64_f32": list(tuned),
                "autotuned_pair_form_f64_f32_outer": list(forms)}
    # end to end through the public API: host (pinned) F in, host U out, right
    # after the device-timed solves (same clocks and the same cached graph)
    F_host = torch.tensor(F_np, dtype=torch.float64).pin_memory()
    U_host = torch.empty_like(F_host).pin_memory()

    def run_e2e():
        # the C-ABI call on host blocks: F read and U written in pinned host
        # memory by the library's kernels, the solve in between
        e2e_t = []
        for i in range(max(1, min(args.steps, 3)) + 1):
            flush.zero_()
            torch.cuda.synchronize()
            t_a = time.perf_counter()
            L.sg_solve_host(h, F_host, hsc_opts, U_host)
            torch.cuda.synchronize()
            if i > 0:
                e2e_t.append((time.perf_counter() - t_a) * 1e3)
        return float(np.mean(e2e_t))

    # headline: mixed HSC-PCG
    with ClockSampler(dev.index if dev.index is not None else 0) as clk:
        ts, st_h, _ = timed_solves(hsc_opts, args.steps, args.warmup)
        e2e_ms = run_e2e()
    ms = float(np.mean(ts))
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    # validation solve (untimed): the true FP64 residual of the same HSC solve
    _, st_true = L.sg_solve(h, F, L.solve_opts(hsc_opts.prec, precond=L.SG_PREC_HSC, tol=1e-8, maxit=500,
                                               check_true_residual=1), U)
    # the solution's residual by the oracle (FP64, host cores; the solve is not timed)
    oracle_res = None
    if rank == 0 and not args.no_cpu_baseline:
        oracle_res = oracle_residual(prob, p, F_np, U.cpu().numpy())
    # comparators on the same GPU, each precision with each preconditioner, so
    # that the speed-up splits into preconditioner and precision: the metric's
    # own comparator is the all-FP64 mean-based PCG
    cmp_steps = max(1, min(args.steps, 2))
    comparators = {}
    for key, opts in (("mean_fp64", mean_opts), ("hsc_fp64", hsc64_opts), ("mean_mixed", mean32_opts),
                      ("hsc_mixed_fp64_products", hsc_f64prod_opts)):
        ts_c, st_c, _ = timed_solves(opts, cmp_steps, 1)
        comparators[key] = {"ms": float(np.mean(ts_c)), "iterations": st_c.iterations, "rel_res": st_c.rel_res,
                            "kappa_est": st_c.kappa_est, "step_ms": ts_c}
    comparators["hsc_mixed"] = {"ms": ms, "iterations": st_h.iterations, "rel_res": st_h.rel_res,
                                "kappa_est": st_h.kappa_est}
    ms_mean = comparators["mean_fp64"]["ms"]

    # kernels per solve: graph replays launch no host calls, so count them on a
    # second handle in eager mode, which runs the same kernels from host-driven loops
    os.environ["SGHSC_EAGER"] = "1"
    h_e = L.SGProblem.from_inputs(prob, p)
    os.environ.pop("SGHSC_EAGER")
    L.sg_autotune(h_e)
    L.sg_solve(h_e, F, hsc_opts, U)
    l0 = L._lib.LIB.sg_kernel_launches()
    L.sg_solve(h_e, F, hsc_opts, U)
    launches = L._lib.LIB.sg_kernel_launches() - l0
    h_e.close()
    del h_e

    # SG matvec roofline: K1 timed alone with events on the launching stream
    def time_apply(dtype, reps=10, df64=False):
        Ut = torch.tensor(S.random_block(n, P, seed=1205), dtype=dtype, device=dev)
        Yt = torch.empty(Ut.shape, dtype=torch.float64 if df64 else dtype, device=dev)
        for _ in range(3):
            L.sg_apply(h, Ut, Yt, df64=df64)
        times = []
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            L.sg_apply(h, Ut, Yt, df64=df64)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        del Ut, Yt
        return float(np.mean(times))

    k1_64 = time_apply(torch.float64)
    k1_32 = time_apply(torch.float32)
    k1_df = time_apply(torch.float32, df64=True)
    hbm, hbm_src = _peaks()
    fp64_peak = L.sg_measure_alu_peak(L.SG_F64) / 1e12      # TFLOP/s, timed alone (burst)
    fp32_peak = L.sg_measure_alu_peak(L.SG_F32) / 1e12
    b64 = sg_matvec_bytes(n, nnz, M, P, 8)
    b32 = sg_matvec_bytes(n, nnz, M, P, 4)
    bdf = sg_matvec_bytes_df(n, nnz, M, P)
    fl = sg_matvec_flops(n, nnz, M, p, P, n_m)
    df_peak = fp32_peak / DF_OPS_PER_MAC
    matvec = {
        "fp64": {"ms": k1_64, "GB_s": b64 / k1_64 / 1e6, "TFLOP_s": fl / k1_64 / 1e9, "bytes": b64, "flops": fl,
                 "frac_fp64_alu_measured": fl / k1_64 / 1e9 / fp64_peak, "frac_hbm": b64 / k1_64 / 1e6 / hbm},
        "fp32": {"ms": k1_32, "GB_s": b32 / k1_32 / 1e6, "TFLOP_s": fl / k1_32 / 1e9, "bytes": b32, "flops": fl,
                 "frac_fp32_alu_measured": fl / k1_32 / 1e9 / fp32_peak, "frac_hbm": b32 / k1_32 / 1e6 / hbm},
        "df64": {"ms": k1_df, "GB_s": bdf / k1_df / 1e6, "TFLOP_s": fl / k1_df / 1e9, "bytes": bdf, "flops": fl,
                 "frac_df64_alu": fl / k1_df / 1e9 / df_peak, "frac_hbm": bdf / k1_df / 1e6 / hbm,
                 "note": "FP32 U, double-float sums, FP64 Y: the product of the outer CG step (k_df_pairs)"},
        "hbm_peak_GB_s": hbm, "hbm_peak_source": hbm_src,
        "fp64_alu_peak_TFLOP_s": fp64_peak, "fp32_alu_peak_TFLOP_s": fp32_peak,
        "df64_alu_peak_TFLOP_s": df_peak,
    }
    # the dominant kernel of the timed solve: the double-float SG product of
    # the outer CG step (its product timed alone through sg_apply, the same
    # kernel body with a plain epilogue)
    roofline = {"kernel": "k_df_pairs (double-float SG product of the outer CG step; timed alone as sg_apply "
                          "SG_F32_ACCDF64)", "bound": "alu",
                "achieved": fl / k1_df / 1e9, "peak": df_peak, "unit": "TFLOP/s",
                "frac": (fl / k1_df / 1e9) / df_peak, "traffic": DF_TRAFFIC.get(args.workload),
                "algorithmic_bytes": bdf, "algorithmic_flops": fl,
                "peak_source": f"measured FP32 FMA-chain rate (sg_measure_alu_peak, timed alone, of measured) / "
                               f"{DF_OPS_PER_MAC} FP32 operations per double-float multiply-add"}


    out = {
        "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 outer CG, df64 (FP32-pair) outer/top-level products, f32 inner", "data": "synthetic (seeded Q1 + exponential-covariance KL, f = 1)",
        "config": workload_config(cfg, world),
        "autotune": {"threads_f64_f32": list(tuned), "pair_form_f64_f32_outer": list(forms),
                     "inner_solver_by_width": inner_paths},
        "hsc": {"ms": ms, "iterations": st_h.iterations, "true_rel_res": st_true.true_rel_res,
                "oracle_rel_res": oracle_res, "arithmetic": "FP32 inner solves and level products < p; outer CG "
                "FP64; outer SG product and level-p products in double-float (df64) on the FP32 units",
                "kappa_est": st_h.kappa_est, "inner_iters_total": st_h.inner_iters_total,
                "inner_iters_max": st_h.inner_iters_max, "step_ms": ts},
        "mean_fp64": {"ms": ms_mean, "iterations": comparators["mean_fp64"]["iterations"],
                      "rel_res": comparators["mean_fp64"]["rel_res"],
                      "kappa_est": comparators["mean_fp64"]["kappa_est"], "speedup_hsc_vs_mean": ms_mean / ms},
        "comparators": comparators,
        "speedups": {"hsc_mixed_vs_mean_fp64": ms_mean / ms,
                     "preconditioner_fp64 (mean_fp64 / hsc_fp64)": ms_mean / comparators["hsc_fp64"]["ms"],
                     "preconditioner_mixed (mean_mixed / hsc_mixed)": comparators["mean_mixed"]["ms"] / ms,
                     "precision_hsc (hsc_fp64 / hsc_mixed)": comparators["hsc_fp64"]["ms"] / ms,
                     "precision_mean (mean_fp64 / mean_mixed)": ms_mean / comparators["mean_mixed"]["ms"],
                     "double_float_products (hsc_mixed_fp64_products / hsc_mixed)":
                         comparators["hsc_mixed_fp64_products"]["ms"] / ms},
        "sg_matvec": matvec,
        "roofline": roofline,
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": int(F_host.numel() * 8),
                "d2h_bytes_per_step": int(U_host.numel() * 8)},
        "gpu_launches": int(launches) * args.steps,
        "gpu_launches_per_step": int(launches),
        "gpu_launches_note": "libsghsc kernels in the timed region: per solve (library launch counter on the same "
                             "solve run in eager mode; the timed solves replay them as one CUDA graph) x steps",
        "clocks": clk.summary(),
        "setup_s": setup_s,
    }
    if cfg.get("grad"):
        out["grad_batch"] = run_grad_batch(cfg, args, dev, flush, hsc_opts)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(cfg, iterations=st_h.iterations)
    return out


def run_grad_batch(cfg, args, dev, flush, opts):
    """The gradient workload: Q and dQ/dtheta (theta = mean coefficient, sigma,
    sqrt(lambda_k) scales) for 16 seeded parameter sets, the forward and the
    adjoint solves of all sets batched on the device (SGGradBatch: one graph
    launch each, then the K7 contraction per set), against the same sets one
    after another through the autograd Function. Wall-clock ms per batch with
    the device synchronised on both sides (the call returns results to the
    host)."""
    import paper_1205_1864_gb300 as L
    import torch
    count = 16
    unit = S.make_unit_problem(cfg["ne"], cfg["M"], cfg["corr_len"])
    base_s = S.theta_of(S.make_problem(cfg["ne"], cfg["M"], 1.0, cfg["corr_len"]))[2:]
    sets = S.draw_grad_params(cfg["M"], count)
    thetas = np.array([np.concatenate([[d["a_mean"], d["sigma"]], base_s * d["sqrt_lambda_scale"]]) for d in sets])
    F = torch.tensor(S.make_rhs(unit, cfg["p"]), dtype=torch.float64, device=dev)
    gb = L.SGGradBatch.from_inputs(unit, cfg["p"], count)
    gb.autotune()

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        ts = []
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append((time.perf_counter() - t0) * 1e3)
        return ts

    ts = timed(lambda: gb.value_and_grad(thetas, F, opts), args.steps, args.warmup)
    Q, G = gb.value_and_grad(thetas, F, opts)
    gb.close()
    h = L.SGProblem.from_inputs(unit, cfg["p"])
    L.sg_autotune(h)
    ts_seq = timed(lambda: L.sg_qoi_value_and_grad_batch(h, thetas, F, opts), 1, 1)
    h.close()
    return {"sets": count, "params_per_set": cfg["M"] + 2, "ms": float(np.mean(ts)), "step_ms": ts,
            "sequential_autograd_ms": ts_seq[0], "speedup_batch_vs_sequential": ts_seq[0] / float(np.mean(ts)),
            "Q_range": [float(Q.min()), float(Q.max())], "grad_norm_max": float(G.abs().max())}


def oracle_residual(prob, p, F, U):
    """||F - A U|| / ||F|| by the FP64 oracle, blocks of rows on a thread pool."""
    from concurrent.futures import ThreadPoolExecutor

    from oracle import chaos, sg_operator as so
    A = so.kl_matrices(prob.rowptr, prob.colidx, prob.vals)
    G = chaos.g_matrices(prob.M, p)
    n, blk = F.shape[0], 8192

    def part(s0):
        rows = np.arange(s0, min(s0 + blk, n))
        R = F[rows] - so.sg_apply_rows(A, G, U, rows)
        return float(np.sum(R * R))

    with ThreadPoolExecutor(host_cores()) as ex:
        ss = sum(ex.map(part, range(0, n, blk)))
    return float(np.sqrt(ss) / np.linalg.norm(F))


def _hsc_opts(L, check=0):
    return L.solve_opts(L.prec_opts(precision=L.SG_F32, top_level_f64=1, inner_tol=1e-2, df64=1),
                        precond=L.SG_PREC_HSC, tol=1e-8, maxit=500, check_true_residual=check)


def _events_time(fn, stream, flush):
    import torch
    flush.zero_()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1), r


def run_batch(args, rank, world, dev):
    """The batched workload: each rank solves its share of the 64 seeded
    systems (longest-processing-time split, no data-path collective) with one
    graph launch per step; the SG-product block size of every system is picked
    by the autotuner first."""
    import torch

    import paper_1205_1864_gb300 as L
    from paper_1205_1864_gb300 import shard
    cfg = WORKLOADS[args.workload]
    cfgs = S.draw_batch_configs(cfg["count"], seed=cfg["seed"])
    costs = [shard.system_cost(c["ne"], c["M"], c["p"]) for c in cfgs]
    mine = shard.my_systems(costs, rank, world)
    t0 = time.time()
    probs, hs, Fs, tuned = [], [], [], []
    for i in mine:
        c = cfgs[i]
        prob = S.make_problem(c["ne"], c["M"], c["sigma"], c["corr_len"])
        h = L.SGProblem.from_inputs(prob, c["p"])
        tuned.append(L.sg_autotune(h))
        probs.append(prob)
        hs.append(h)
        Fs.append(torch.tensor(S.make_rhs(prob, c["p"]), dtype=torch.float64, device=dev))
    setup_s = time.time() - t0
    Us = [torch.empty_like(F) for F in Fs]
    batch = L.SGBatch(hs)
    opts = _hsc_opts(L)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    unknowns = sum(h.n * h.P for h in hs)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ts, last = [], None
        for _ in range(steps):
            t, last = _events_time(fn, stream, flush)
            ts.append(t)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        return ts, last

    solve_batch = lambda: batch.solve(Fs, opts, Us)[1]
    if args.profile:
        ts, st = timed(solve_batch, args.steps, args.warmup)
        return {"profile": True, "workload": cfg["name"], "ms": float(np.mean(ts)),
                "iterations": [s.iterations for s in st]}
    with ClockSampler(dev.index if dev.index is not None else 0) as clk:
        ts, st = timed(solve_batch, args.steps, args.warmup)
    ms = shard.max_over_ranks(float(np.mean(ts)), device=dev)
    # validation (untimed): the true FP64 residual of every system
    _, st_true = batch.solve(Fs, _hsc_opts(L, check=1), Us)
    # comparator: the same systems one sg_solve (one graph launch) after another
    seq = lambda: [L.sg_solve(h, F, opts, U)[1] for h, F, U in zip(hs, Fs, Us)]
    ts_seq, _ = timed(seq, max(1, min(args.steps, 3)), 1)
    ms_seq = float(np.mean(ts_seq))
    # kernels per step, counted on eager twins of each handle (same kernels, host-driven loops)
    launches = 0
    for prob, i in zip(probs, mine):
        os.environ["SGHSC_EAGER"] = "1"
        he = L.SGProblem.from_inputs(prob, cfgs[i]["p"])
        os.environ.pop("SGHSC_EAGER")
        L.sg_autotune(he)
        F = Fs[mine.index(i)]
        L.sg_solve(he, F, opts)
        l0 = L._lib.LIB.sg_kernel_launches()
        L.sg_solve(he, F, opts)
        launches += L._lib.LIB.sg_kernel_launches() - l0
        he.close()
    # K1 roofline on the largest system of this rank
    big = max(range(len(hs)), key=lambda j: hs[j].n * hs[j].P)
    hb = hs[big]
    Ut = torch.tensor(S.random_block(hb.n, hb.P, seed=1205), dtype=torch.float64, device=dev)
    Yt = torch.empty_like(Ut)
    for _ in range(3):
        L.sg_apply(hb, Ut, Yt)
    k1 = float(np.mean([_events_time(lambda: L.sg_apply(hb, Ut, Yt), stream, flush)[0] for _ in range(20)]))
    M_b, p_b = hb.M, cfgs[mine[big]]["p"]
    fl = sg_matvec_flops(hb.n, hb.nnz, M_b, p_b, hb.P, int(2 * M_b * math.comb(M_b + p_b - 1, M_b)))
    fp64_peak = L.sg_measure_alu_peak(L.SG_F64) / 1e12
    roofline = {"kernel": f"k_block_matvec<double> (K1 FP64 SG product) on the largest system (n={hb.n}, P={hb.P})",
                "bound": "alu", "achieved": fl / k1 / 1e9, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": (fl / k1 / 1e9) / fp64_peak, "traffic": None,
                "peak_source": "measured: FP64 FMA-chain kernel (sg_measure_alu_peak) on this GPU, timed alone, "
                               "of measured"}
    # end to end through the public API: host (pinned) right-hand sides in, solutions out
    F_host = [F.cpu().pin_memory() for F in Fs]
    U_host = [torch.empty_like(F).pin_memory() for F in F_host]
    e2e_t = []
    for k in range(max(1, min(args.steps, 3)) + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t_a = time.perf_counter()
        batch.solve_host(F_host, opts, U_host)   # host blocks in and out, moved by the library's kernels
        torch.cuda.synchronize()
        if k > 0:
            e2e_t.append((time.perf_counter() - t_a) * 1e3)
    e2e_ms = shard.max_over_ranks(float(np.mean(e2e_t)), device=dev)
    nbytes = sum(F.numel() * 8 for F in F_host)
    out = {
        "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": False, "scaling": "strong", "vs_baseline": None,
        "dtype": "f64 outer CG, df64 (FP32-pair) outer/top-level products, f32 inner", "data": "synthetic (seeded Q1 + exponential-covariance KL, f = 1)",
        "config": workload_config(cfg, world),
        "batch": {"ms": ms, "step_ms": ts, "systems_this_rank": len(mine), "unknowns_this_rank": unknowns,
                  "iterations": [s.iterations for s in st],
                  "status": [s.status for s in st], "max_true_rel_res": max(s.true_rel_res for s in st_true),
                  "autotuned_threads_f64_f32": tuned, "sequential_ms": ms_seq,
                  "speedup_batch_vs_sequential": ms_seq / float(np.mean(ts))},
        "roofline": roofline,
        "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": int(nbytes), "d2h_bytes_per_step": int(nbytes)},
        "gpu_launches": int(launches) * args.steps,
        "gpu_launches_per_step": int(launches),
        "gpu_launches_note": "libsghsc kernels in the timed region: per batch step (launch counter on eager twins of "
                             "every handle; the timed step replays them as one CUDA graph) x steps",
        "clocks": clk.summary(),
        "setup_s": setup_s,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_batch(cfgs, [s.iterations for s in st])
    batch.close()
    return out


# --------------------------------------------------------------------------
# CPU baseline: the FP64 oracle as it stands, on all host cores
# --------------------------------------------------------------------------
#
# One outer HSC-FCG iteration of the oracle is an SG product (oracle
# sg_operator), the 2p level products of Algorithm 1 (sg_operator.level_apply)
# and n_ds = 2 (P - 1) + 1 inner column solves (krylov.pcg_columns with one
# gmg.vcycle per step, tolerance 1e-2: the algorithm the GPU runs). Each of
# them is independent across spatial rows (products) or columns (inner solves),
# so the host's cores each take a share: a pool of spawned processes, one per
# core, each holding the problem. The sample times, on every core at once, one
# block of rows of the products and one inner column solve, and scales them to
# the whole iteration and to the solve's iteration count.

_CPU = {}


def _cpu_init(cfg):
    from oracle import chaos, gmg, sg_operator as so
    prob = S.make_problem(cfg["ne"], cfg["M"], cfg["sigma"], cfg["corr_len"])
    A = so.kl_matrices(prob.rowptr, prob.colidx, prob.vals)
    G = chaos.g_matrices(cfg["M"], cfg["p"])
    _, off = chaos.multi_indices(cfg["M"], cfg["p"])
    P = G[0].shape[0]
    # inputs: untouched zero pages until a row block reads them (the products'
    # time does not depend on the values); one contiguous block per degree level
    _CPU.update(A=A, G=G, off=off, n=prob.n, P=P, p=cfg["p"], lv=gmg.hierarchy(A[0], cfg["ne"]),
                U=np.zeros((prob.n, P)), Ul=[np.zeros((prob.n, off[l + 1] - off[l])) for l in range(cfg["p"] + 1)])


def _cpu_products(task):
    """Wall time of the SG product and of the 2p level products on one block of rows."""
    from oracle import sg_operator as so
    start, count = task
    c = _CPU
    rows = np.arange(start, min(start + count, c["n"]))
    t0 = time.perf_counter()
    so.sg_apply_rows(c["A"], c["G"], c["U"], rows)
    t1 = time.perf_counter()
    off, p = c["off"], c["p"]
    for l in range(1, p + 1):
        for lo, li in ((l - 1, l), (l, l - 1)):
            so.level_apply(c["A"], c["G"], off, lo, li, c["Ul"][li], rows=rows)
    return t1 - t0, time.perf_counter() - t1


def _cpu_column(seed):
    """Wall time and iterations of one inner column solve (V-cycle PCG, tol 1e-2)."""
    from oracle import gmg, krylov
    c = _CPU
    b = np.random.default_rng(seed).uniform(-1.0, 1.0, size=(c["n"], 1))
    A0, lv = c["A"][0], c["lv"]
    t0 = time.perf_counter()
    _, it = krylov.pcg_columns(lambda v: A0 @ v, b, lambda r: gmg.vcycle(lv, r, nu=2, omega=0.8), tol=1e-2,
                               maxit=200)
    return time.perf_counter() - t0, int(it[0])


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


class CpuOracle:
    """A pool of spawned processes, one per host core, each holding one
    problem of the workload for the oracle's timed samples."""

    def __init__(self, cfg, cores=None):
        import multiprocessing as mp
        self.cfg = cfg
        self.cores = cores or host_cores()
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_cpu_init, initargs=(cfg,))
        n = (cfg["ne"] - 1) ** 2
        self.n = n
        self.P = math.comb(cfg["M"] + cfg["p"], cfg["M"])

    def close(self):
        self.pool.terminate()
        self.pool.join()

    def sample(self, iterations, rows_per_core=None):
        """One bounded sample: every core times one block of rows of the
        products and one inner column solve; returns the estimate of the
        oracle's whole solve (ms) and what was sampled."""
        cores, n, P = self.cores, self.n, self.P
        B = rows_per_core or max(16, min(n // cores, max(1, 2_000_000 // max(P, 1))))
        tasks = [((i * B) % max(n - B, 1), B) for i in range(cores)]
        t0 = time.perf_counter()
        prod = self.pool.map(_cpu_products, tasks, chunksize=1)
        t1 = time.perf_counter()
        cols = self.pool.map(_cpu_column, list(range(cores)), chunksize=1)
        t2 = time.perf_counter()
        # every core busy at once: the wall time of one round covers cores blocks / columns
        rounds_rows = n / (B * cores)
        t_apply = max(a for a, _ in prod) * rounds_rows
        t_levels = max(b for _, b in prod) * rounds_rows
        n_ds = 2 * (P - 1) + 1
        t_inner = (t2 - t1) * math.ceil(n_ds / cores)
        per_iter = t_apply + t_levels + t_inner
        value_ms = per_iter * max(iterations, 1) * 1e3
        its = sorted({i for _, i in cols})
        desc = (f"FP64 oracle on {cores} host cores (one spawned process per core): per core {B} rows of the SG "
                f"product and of the 2p level products of Algorithm 1 ({t1 - t0:.2f} s wall) and one inner "
                f"V-cycle-PCG column solve at tol 1e-2 ({t2 - t1:.2f} s wall, {its} iterations); scaled to {n} "
                f"rows and n_ds = {n_ds} column solves per HSC application: {per_iter:.2f} s per outer "
                f"iteration (product {t_apply:.2f} s, level products {t_levels:.2f} s, inner solves "
                f"{t_inner:.2f} s) x {iterations} iterations")
        return value_ms, desc


def cpu_baseline(cfg, iterations, oracle=None):
    own = oracle is None
    oracle = oracle or CpuOracle(cfg)
    try:
        t0 = time.perf_counter()
        v, desc = oracle.sample(iterations)
        return {"value": v, "unit": "ms", "cores": oracle.cores, "kind": "oracle", "sample": desc,
                "wall_s": time.perf_counter() - t0}
    finally:
        if own:
            oracle.close()


def cpu_baseline_batch(cfgs, iterations):
    """The oracle on a bounded sample of the batch: per mesh size, the first
    system of that size in draw order, sampled on all host cores for one outer
    iteration; every system's full solve is then estimated from its class's
    time per unit of cost, times its own cost and GPU iteration count."""
    from paper_1205_1864_gb300 import shard
    costs = [shard.system_cost(c["ne"], c["M"], c["p"]) for c in cfgs]
    rate, sampled = {}, []
    t0 = time.perf_counter()
    cores = host_cores()
    for ne in sorted({c["ne"] for c in cfgs}):
        i = next(j for j, c in enumerate(cfgs) if c["ne"] == ne)
        c = cfgs[i]
        cb = cpu_baseline(dict(name=f"system {i}", **c), iterations=1)
        rate[ne] = cb["value"] / costs[i]
        sampled.append(f"#{i} ({ne}x{ne}, M={c['M']}, p={c['p']}): {cb['value']:.0f} ms/iteration")
        cores = cb["cores"]
    value = sum(rate[c["ne"]] * costs[j] * max(iterations[j], 1) for j, c in enumerate(cfgs))
    return {"value": value, "unit": "ms", "cores": cores, "kind": "oracle",
            "sample": "one outer HSC-FCG iteration of the FP64 oracle per mesh size, sampled on all host cores (" +
                      "; ".join(sampled) + "), scaled per system by cost and GPU iteration count to all systems",
            "wall_s": time.perf_counter() - t0}


def run_reference(args, rank, world):
    """The oracle, as it stands, on the host cores: each step is one bounded
    sample of the workload's solve (see CpuOracle), on rank 0 only."""
    if rank != 0:
        return None
    cfg = WORKLOADS[args.workload]
    vals = []
    if cfg.get("batch"):
        cfgs = S.draw_batch_configs(cfg["count"], seed=cfg["seed"])
        for i in range(args.warmup + args.steps):
            cb = cpu_baseline_batch(cfgs, [6] * len(cfgs))   # ~6 HSC-FCG iterations at 1e-8
            if i >= args.warmup:
                vals.append(cb["value"])
    else:
        oracle = CpuOracle(cfg)
        try:
            for i in range(args.warmup + args.steps):
                cb = cpu_baseline(cfg, iterations=cfg["hsc_iterations"], oracle=oracle)
                if i >= args.warmup:
                    vals.append(cb["value"])
        finally:
            oracle.close()
    v = float(np.mean(vals))
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Q1 + exponential-covariance KL, f = 1)",
            "config": workload_config(cfg, world),
            "cpu_baseline": {"value": v, "unit": "ms", "cores": cb["cores"], "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _golden(name):
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


def run_tables(dev):
    """The paper's Tables 1-4 (Sec. 6) on the GPU: outer iterations and Lanczos
    condition estimates of flexible CG to 1e-8 with M_m, M_bGS and M_HS (all
    FP64, inner PCG with the diagonal M_0 to 1e-8), next to the printed values."""
    import paper_1205_1864_gb300 as L
    import torch
    code = {"mean": L.SG_PREC_MEAN, "bgs": L.SG_PREC_BGS, "hsc": L.SG_PREC_HSC}
    # (name, fixture, (mesh, M, p, CoV) of a row, column of M_m's iteration count)
    specs = [("table1_vary_N", "sec6_table1_vary_N_full.txt", lambda r: (10, int(r[0]), 4, 0.5), 4),
             ("table2_vary_P", "sec6_table2_vary_P.txt", lambda r: (10, 4, int(r[0]), 0.5), 4),
             ("table3_vary_cov", "sec6_table3_vary_cov_full.txt", lambda r: (10, 4, 4, r[0] / 100.0), 3),
             ("table4_vary_h", "sec6_table4_vary_h.txt", lambda r: (int(r[0]), 4, 4, 0.5), 4)]
    out = {"profile": "tables", "setting": "Sec. 6: k0 = 1, L = 0.5, f = 1, sigma = CoV/sqrt(3), FP64, inner PCG "
                                           "with diagonal M_0 to 1e-8, outer flexible CG to 1e-8"}
    for name, fname, setting, c0 in specs:
        rows = []
        for r in _golden(fname):
            ne, M, p, cov = setting(r)
            prob = S.make_problem(ne, M, cov / math.sqrt(3.0), 0.5)
            h = L.SGProblem.from_inputs(prob, p)
            F = torch.tensor(S.make_rhs(prob, p), dtype=torch.float64, device=dev)
            row = {"key": r[0], "ndof_interior": h.n * h.P}
            for k, col in (("mean", c0), ("bgs", c0 + 2), ("hsc", c0 + 4)):
                o = L.solve_opts(L.prec_opts(precision=L.SG_F64, m0=L.SG_M0_DIAG, inner_tol=1e-8, inner_maxit=1000),
                                 precond=code[k], tol=1e-8, maxit=1000)
                _, st = L.sg_solve(h, F, o)
                row[k] = [st.iterations, round(st.kappa_est, 4)]
                row[k + "_paper"] = [int(r[col]), r[col + 1]]
            rows.append(row)
            h.close()
        out[name] = rows
    # Tables 6-9: the gPC expansion of a lognormal coefficient (Hermite chaos, coefficient degree 2p),
    # M_m and M_HS (Algorithm 1 with the nested D_l solves, level_tol 1e-8)
    specs = [("table6_lognormal_vary_N", "sec6_table6_lognormal_vary_N.txt", lambda r: (10, int(r[0]), 4, 1.0), 4),
             ("table7_lognormal_vary_P", "sec6_table7_lognormal_vary_P.txt", lambda r: (10, 4, int(r[0]), 1.0), 4),
             ("table8_lognormal_vary_cov", "sec6_table8_lognormal_vary_cov.txt", lambda r: (10, 4, 4, r[0] / 100.0),
              3),
             ("table9_lognormal_vary_h", "sec6_table9_lognormal_vary_h.txt", lambda r: (int(r[0]), 4, 4, 1.0), 4)]
    for name, fname, setting, c0 in specs:
        rows = []
        for r in _golden(fname):
            ne, M, p, cov = setting(r)
            prob = S.make_lognormal_problem(ne, M, cov, 0.5, 2 * p)
            h = L.SGProblem.from_inputs(prob, p)
            F = torch.tensor(S.make_rhs(prob, p), dtype=torch.float64, device=dev)
            row = {"key": r[0], "ndof_interior": h.n * h.P, "coef_terms": h.nterm}
            for k, col in (("mean", c0), ("hsc", c0 + 4)):
                o = L.solve_opts(L.prec_opts(precision=L.SG_F64, m0=L.SG_M0_DIAG, inner_tol=1e-8, level_tol=1e-8,
                                             level_maxit=2000, inner_maxit=1000),
                                 precond=code[k], tol=1e-8, maxit=1000)
                _, st = L.sg_solve(h, F, o)
                row[k] = [st.iterations, round(st.kappa_est, 4)]
                row[k + "_paper"] = [int(r[col]), r[col + 1]]
            row["bgs_paper"] = [int(r[c0 + 2]), r[c0 + 3]]
            rows.append(row)
            h.close()
        out[name] = rows
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cfg5", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ne", type=int, default=None,
                    help="mesh override (elements per side, a power of two) for profiling a workload's kernel "
                         "shapes on a smaller case; the name gets an @ne suffix")
    ap.add_argument("--profile", nargs="?", const="solve", default=None,
                    choices=["solve", "apply", "levels", "inner", "tables"],
                    help="solve: only the warm-up and timed HSC solves; apply: only the SG product, FP64, "
                         "FP32 and FP32 with double-float sums; levels: every level product in each arithmetic; "
                         "inner: only the batched inner PCG on the widest level (for ncu captures); "
                         "tables: the paper's Tables 1-4 on the GPU next to the printed values; "
                         "prints one short line")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.ne is not None:
        w = dict(WORKLOADS[args.workload])
        if w.get("batch"):
            ap.error("--ne applies to single-system workloads")
        w["ne"] = args.ne
        w["name"] = f"{w['name']}@ne{args.ne}"
        WORKLOADS[args.workload] = w
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=dev)
    if args.profile == "tables":
        out = run_tables(dev)
    else:
        out = run_batch(args, rank, world, dev) if WORKLOADS[args.workload].get("batch") else \
            run_ours(args, rank, world, dev)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
