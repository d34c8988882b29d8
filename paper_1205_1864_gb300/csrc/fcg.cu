// K5: the outer flexible conjugate gradient method on eq. (global-system)
// (Sec. 5: flexible CG for the variable HSC preconditioner; Sec. 6: relative
// residual 1e-8 and the Lanczos condition estimate). Everything here is FP64:
// residual, search directions, dot products and the SG product of K1.
//
// The iteration is a CUDA graph WHILE node: the CG scalars live on the device
// (the last block of each reduction kernel updates them) and the update
// kernel sets the loop condition, so a whole solve is one graph launch with
// no host round trip; the host reads the statistics once at the end.
//
// Loop body (precondition first, so the loop test is the residual test):
//   z = M r                                  (HSC, mean-based or identity)
//   beta = z.(r - r_old)/rho_old (flexible) or z.r/rho_old; rho = z.r
//   p = z + beta p;  q = A p;  alpha = rho / p.q       (fused in K1)
//   x += alpha p;  r -= alpha q;  test ||r|| / ||f|| and the iteration cap
#include <chrono>
#include <cmath>
#include <cstdio>
#include <vector>

#include "graph.cuh"
#include "sghsc_internal.cuh"
#include "vec.cuh"

namespace sghsc {

int ensure_outer(sg_problem* h) {
  if (!h->fr) {
    if (h->capturing) {
      set_error("outer buffers must be allocated before graph capture");
      return SG_ERR_UNSUPPORTED;
    }
    const size_t bytes = (size_t)h->n * h->P * sizeof(double);
    for (double** b : {&h->fF, &h->fx, &h->fr, &h->fz, &h->fpA, &h->fpB, &h->fq})
      SG_TRY_CUDA(cudaMalloc((void**)b, bytes));
    SG_TRY_CUDA(cudaMalloc((void**)&h->osc, SC_COUNT * sizeof(double)));
    SG_TRY_CUDA(cudaMallocHost((void**)&h->osc_host, SC_COUNT * sizeof(double)));
    SG_TRY_CUDA(cudaMalloc((void**)&h->octl, sizeof(OuterCtl)));
    SG_TRY_CUDA(cudaMemset(h->octl, 0, sizeof(OuterCtl)));
    SG_TRY_CUDA(cudaMalloc((void**)&h->hist_alpha, (SG_MAX_HIST + 1) * sizeof(double)));
    SG_TRY_CUDA(cudaMalloc((void**)&h->hist_beta, (SG_MAX_HIST + 1) * sizeof(double)));
    SG_TRY_CUDA(cudaMalloc((void**)&h->hist_res, (SG_MAX_HIST + 2) * sizeof(double)));
    SG_TRY_CUDA(cudaMemset(h->fpA, 0, bytes));
    SG_TRY_CUDA(cudaMemset(h->fpB, 0, bytes));
    SG_TRY_CUDA(cudaMemset(h->fq, 0, bytes));
  }
  // partial sums: the K1 grid (<= 8 blocks per SM) and the vector grid both fit
  const int need = std::max(h->num_sms * 16, 152 * 8);
  if (!h->opart || h->opart_blocks < need) {
    if (h->capturing) {
      set_error("outer buffers must be allocated before graph capture");
      return SG_ERR_UNSUPPORTED;
    }
    if (h->opart) {
      clear_graphs(h);   // captured graphs hold the old partial-sum buffer
      SG_TRY_CUDA(cudaDeviceSynchronize());
    }
    cudaFree(h->opart);
    h->opart = nullptr;   // a failed allocation leaves no stale buffer behind
    h->opart_blocks = 0;
    SG_TRY_CUDA(cudaMalloc((void**)&h->opart, (size_t)need * 2 * sizeof(double)));
    h->opart_blocks = need;
  }
  return SG_OK;
}

// Largest and smallest eigenvalue of the symmetric tridiagonal (d, e) by
// Sturm-sequence bisection.
static int sturm_count(const std::vector<double>& d, const std::vector<double>& e, double x) {
  int cnt = 0;
  double q = 1.0;
  for (size_t i = 0; i < d.size(); ++i) {
    const double e2 = i ? e[i - 1] * e[i - 1] : 0.0;
    q = d[i] - x - (i ? e2 / (q == 0.0 ? 1e-300 : q) : 0.0);
    if (q < 0) ++cnt;
  }
  return cnt;
}

static double tridiag_eig(const std::vector<double>& d, const std::vector<double>& e, int k) {
  double lo = 1e300, hi = -1e300;
  for (size_t i = 0; i < d.size(); ++i) {
    const double r = (i ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < d.size() ? std::fabs(e[i]) : 0.0);
    lo = std::min(lo, d[i] - r);
    hi = std::max(hi, d[i] + r);
  }
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_count(d, e, mid) > k) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// Lanczos estimate (Sec. 6) from the CG coefficients:
// T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1}, T_{j,j+1} = sqrt(beta_j)/alpha_j.
static double lanczos_kappa(const double* alpha, const double* beta, int m) {
  if (m <= 0) return 1.0;
  std::vector<double> d(m), e(std::max(m - 1, 0));
  for (int j = 0; j < m; ++j) {
    d[j] = 1.0 / alpha[j] + (j > 0 ? beta[j - 1] / alpha[j - 1] : 0.0);
    if (j + 1 < m) e[j] = std::sqrt(std::max(beta[j], 0.0)) / alpha[j];
  }
  const double lmin = tridiag_eig(d, e, 0), lmax = tridiag_eig(d, e, m - 1);
  return lmin > 0 ? lmax / lmin : INFINITY;
}

static int precond(sg_problem* h, int kind, const double* r, double* z, const sg_prec_opts& o, cudaStream_t s) {
  if (kind == SG_PREC_HSC) return hsc_apply_impl(h, r, z, o, s);
  if (kind == SG_PREC_MEAN) return mean_apply_impl(h, r, z, o, s);
  if (kind == SG_PREC_BGS) return bgs_apply_impl(h, r, z, o, s);
  SG_TRY_CUDA(cudaMemcpyAsync(z, r, (size_t)h->n * h->P * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return SG_OK;
}

OuterArgs outer_args(sg_problem* h, const sg_solve_opts& o) {
  OuterArgs a;
  a.part = h->opart;
  a.ctl = h->octl;
  a.sc = h->osc;
  a.hist_alpha = h->hist_alpha;
  a.hist_beta = h->hist_beta;
  a.hist_res = h->hist_res;
  a.status = h->status;
  a.flexible = o.flexible;
  a.maxit = std::min(o.maxit, SG_MAX_HIST);
  a.tol = o.tol;
  a.cond = 0;
  a.has_cond = 0;
  a.flag = nullptr;
  return a;
}

// The whole solve, enqueued on a capturing stream.
int enqueue_solve(sg_problem* h, const sg_solve_opts& o, cudaStream_t s) {
  const long long N = (long long)h->n * h->P;
  const int vg = std::min(vec_grid(N), h->opart_blocks);
  OuterArgs a0 = outer_args(h, o);
  auto pre = [&](cudaStream_t ps, const LoopCtl& lc) -> int {
    OuterArgs a = a0;
    a.cond = lc.cond;
    a.has_cond = lc.has_cond;
    a.flag = lc.flag;
    if (o.use_x0) {
      SG_TRY(launch_block_matvec(h, SG_F64, SG_F64, SG_F64, SG_F64, h->fx, h->P, h->P, h->all, true, nullptr, 0, 1.0,
                                 0.0, h->fq, h->P, ps));
      { k_outer_init<<<vg, 256, 0, ps>>>(N, h->fF, h->fq, h->fr, a); ::sghsc::note_launch(); }
    } else {
      SG_TRY_CUDA(cudaMemsetAsync(h->fx, 0, N * sizeof(double), ps));
      { k_outer_init<<<vg, 256, 0, ps>>>(N, h->fF, nullptr, h->fr, a); ::sghsc::note_launch(); }
    }
    SG_CHECK_LAUNCH();
    return SG_OK;
  };
  auto body = [&](cudaStream_t bs, const LoopCtl& lc) -> int {
    OuterArgs a = a0;
    a.cond = lc.cond;
    a.has_cond = lc.has_cond;
    a.flag = lc.flag;
    // with an FP32 preconditioner and df64, the outer product runs in double-float arithmetic
    const bool df = o.precond != SG_PREC_NONE && o.prec.precision == SG_F32 && o.prec.df64;
    // Algorithm 1 and block Gauss-Seidel in FP32 leave z in h->Z32: the dots
    // and the outer product read it there (widened exactly on the fly), so z
    // is never written in FP64
    // (the staged outer product reads z32; the row-per-warp one reads FP64 z)
    const float* z32 = df && (o.precond == SG_PREC_HSC || o.precond == SG_PREC_BGS) &&
                               df_pairs_usable(h, h->all, h->P) ? h->Z32 : nullptr;
    SG_TRY(precond(h, o.precond, h->fr, z32 ? nullptr : h->fz, o.prec, bs));
    if (z32)
      { k_outer_dots32<<<vg, 256, 0, bs>>>(N, z32, h->fr, h->fq, a); ::sghsc::note_launch(); }
    else
      { k_outer_dots<<<vg, 256, 0, bs>>>(N, h->fz, h->fr, h->fq, a); ::sghsc::note_launch(); }
    SG_TRY(launch_outer_matvec(h, a, bs, df, z32));
    { k_outer_update<<<vg, 256, 0, bs>>>(N, h->fpA, h->fpB, h->fq, h->fx, h->fr, a); ::sghsc::note_launch(); }
    SG_CHECK_LAUNCH();
    return SG_OK;
  };
  SG_TRY(capture_while(h, s, pre, body));
  if (o.check_true_residual) {
    SG_TRY(launch_block_matvec(h, SG_F64, SG_F64, SG_F64, SG_F64, h->fx, h->P, h->P, h->all, true, nullptr, 0, 1.0,
                               0.0, h->fq, h->P, s));
    { k_outer_true<<<vg, 256, 0, s>>>(N, h->fF, h->fq, a0); ::sghsc::note_launch(); }
    SG_CHECK_LAUNCH();
  }
  return SG_OK;
}

// The a-priori reduction of Sec. 5 (eq. (global-Schur-system)): flexible CG
// on S_{p-1} u_{p-1} = g_{p-1}, S_{p-1} = A_{p-1} - B_p D_p^{-1} C_p, over the
// n x Pr blocks of levels 0..p-1 (leading dimension Pr = off[p]); then
// u^p = D_p^{-1} (f^p - C_p u_{p-1}). The D_p^{-1} actions inside the operator
// are FP64 inner solves to schur_inner_tol (the reduction assumes exact
// ones). The iteration keeps p in one buffer (fpA) and q in fq; the assembled
// n x P solution ends in fz.
static int enqueue_schur_solve(sg_problem* h, const sg_solve_opts& o, cudaStream_t s) {
  const int P = h->P, p = h->p, n = h->n;
  const int Pr = h->off[p], wp = P - Pr, lo1 = h->off[p - 1], w1 = Pr - lo1;
  const long long N = (long long)n * Pr;
  const int vg = std::min(vec_grid(N), h->opart_blocks);
  sg_prec_opts dop = o.prec;     // the exact-solve stand-in for D_p^{-1}
  dop.precision = SG_F64;
  dop.inner_tol = o.schur_inner_tol;
  dop.inner_fixed_iters = 0;
  dop.inner_maxit = std::max(o.prec.inner_maxit, 1000);
  double* Y = h->R64w;           // n x wp: D_p^{-1} of a level-p block
  double* T = h->T64;            // n x wp: a level-p block
  const OuterArgs a0 = outer_args(h, o);
  auto with = [&](const LoopCtl& lc) {
    OuterArgs a = a0;
    a.cond = lc.cond;
    a.has_cond = lc.has_cond;
    a.flag = lc.flag;
    return a;
  };
  auto pre = [&](cudaStream_t ps, const LoopCtl& lc) -> int {
    const OuterArgs a = with(lc);
    // g = f^{<p} - B_p D_p^{-1} f^p
    SG_TRY(launch_cast(h->fF, SG_F64, P, h->fG, SG_F64, Pr, n, Pr, ps));
    SG_TRY(inner_solve(h, SG_F64, h->fF + Pr, P, SG_F64, Y, wp, SG_F64, wp, dop, ps));
    SG_TRY(launch_block_matvec(h, SG_F64, SG_F64, SG_F64, SG_F64, Y, wp, wp, h->pre[p], false, h->fG + lo1, Pr, -1.0,
                               1.0, h->fG + lo1, Pr, ps));
    SG_TRY_CUDA(cudaMemsetAsync(h->fx, 0, N * sizeof(double), ps));
    { k_outer_init<<<vg, 256, 0, ps>>>(N, h->fG, nullptr, h->fr, a); ::sghsc::note_launch(); }
    SG_CHECK_LAUNCH();
    return SG_OK;
  };
  auto body = [&](cudaStream_t bs, const LoopCtl& lc) -> int {
    const OuterArgs a = with(lc);
    if (o.precond == SG_PREC_HSC) SG_TRY(hsc_apply_lv(h, h->fr, h->fz, o.prec, bs, p - 1, Pr));
    else if (o.precond == SG_PREC_BGS) SG_TRY(bgs_apply_lv(h, h->fr, h->fz, o.prec, bs, p - 1, Pr));
    else if (o.precond == SG_PREC_MEAN) SG_TRY(mean_apply_lv(h, h->fr, h->fz, o.prec, bs, Pr));
    else SG_TRY_CUDA(cudaMemcpyAsync(h->fz, h->fr, N * sizeof(double), cudaMemcpyDeviceToDevice, bs));
    { k_outer_dots<<<vg, 256, 0, bs>>>(N, h->fz, h->fr, h->fq, a); ::sghsc::note_launch(); }
    { k_schur_p<<<vg, 256, 0, bs>>>(N, h->fz, h->fpA, a); ::sghsc::note_launch(); }
    // q = A_{p-1} p - B_p D_p^{-1} C_p p
    SG_TRY(launch_block_matvec(h, SG_F64, SG_F64, SG_F64, SG_F64, h->fpA, Pr, Pr, h->sub, true, nullptr, 0, 1.0, 0.0,
                               h->fq, Pr, bs));
    SG_TRY(launch_block_matvec(h, SG_F64, SG_F64, SG_F64, SG_F64, h->fpA + lo1, Pr, w1, h->post[p], false, nullptr, 0,
                               1.0, 0.0, T, wp, bs));
    SG_TRY(inner_solve(h, SG_F64, T, wp, SG_F64, Y, wp, SG_F64, wp, dop, bs));
    SG_TRY(launch_block_matvec(h, SG_F64, SG_F64, SG_F64, SG_F64, Y, wp, wp, h->pre[p], false, h->fq + lo1, Pr, -1.0,
                               1.0, h->fq + lo1, Pr, bs));
    { k_schur_pq<<<vg, 256, 0, bs>>>(N, h->fpA, h->fq, a); ::sghsc::note_launch(); }
    { k_outer_update<<<vg, 256, 0, bs>>>(N, h->fpA, h->fpA, h->fq, h->fx, h->fr, a); ::sghsc::note_launch(); }
    SG_CHECK_LAUNCH();
    return SG_OK;
  };
  SG_TRY(capture_while(h, s, pre, body));
  // recovery: u^p = D_p^{-1} (f^p - C_p u_{p-1}), assembled with u_{p-1} in fz
  SG_TRY(launch_block_matvec(h, SG_F64, SG_F64, SG_F64, SG_F64, h->fx + lo1, Pr, w1, h->post[p], false, h->fF + Pr, P,
                             -1.0, 1.0, T, wp, s));
  SG_TRY(inner_solve(h, SG_F64, T, wp, SG_F64, h->fz + Pr, P, SG_F64, wp, dop, s));
  SG_TRY(launch_cast(h->fx, SG_F64, Pr, h->fz, SG_F64, P, n, Pr, s));
  if (o.check_true_residual) {
    const long long NF = (long long)n * P;
    SG_TRY(launch_block_matvec(h, SG_F64, SG_F64, SG_F64, SG_F64, h->fz, P, P, h->all, true, nullptr, 0, 1.0, 0.0,
                               h->fq, P, s));
    { k_outer_true<<<std::min(vec_grid(NF), h->opart_blocks), 256, 0, s>>>(NF, h->fF, h->fq, a0); ::sghsc::note_launch(); }
    SG_CHECK_LAUNCH();
  }
  return SG_OK;
}

std::string opts_key(const sg_prec_opts& o) {
  char buf[256];
  snprintf(buf, sizeof buf, "p%d|t%d|tol%.17g|mi%d|fx%d|nu%d|om%.17g|m%d|lt%.17g|lm%d|md%d|df%d", o.precision,
           o.top_level_f64, o.inner_tol, o.inner_maxit, o.inner_fixed_iters, o.nu, o.omega, o.m0, o.level_tol,
           o.level_maxit, o.md_m0, o.df64);
  return buf;
}

int solve_prepare(sg_problem* h, const sg_solve_opts& o) {
  SG_TRY(ensure_outer(h));
  if (o.precond != SG_PREC_NONE) SG_TRY(prepare_precond(h, o.precond, o.prec));
  if (o.schur_reduced) {
    // FP64 inner solves of the level-p blocks and their buffers, the reduced right-hand side
    sg_prec_opts dop = o.prec;
    dop.precision = SG_F64;
    SG_TRY(prepare_precond(h, SG_PREC_HSC, dop));
    if (!h->fG) {
      if (h->capturing) {
        set_error("outer buffers must be allocated before graph capture");
        return SG_ERR_UNSUPPORTED;
      }
      SG_TRY_CUDA(cudaMalloc((void**)&h->fG, (size_t)h->n * h->off[h->p] * sizeof(double)));
    }
  }
  return SG_OK;
}

std::string solve_key(const sg_solve_opts& o) {
  char key[512];
  snprintf(key, sizeof key, "solve|k%d|%s|tol%.17g|mi%d|fl%d|x0%d|tr%d|sr%d|st%.17g", o.precond,
           o.precond == SG_PREC_NONE && !o.schur_reduced ? "-" : opts_key(o.prec).c_str(), o.tol, o.maxit, o.flexible,
           o.use_x0, o.check_true_residual, o.schur_reduced, o.schur_reduced ? o.schur_inner_tol : 0.0);
  return key;
}

// Copy the right-hand side (and the initial guess) into the handle's buffers.
int solve_stage_in(sg_problem* h, const double* F, const double* U, const sg_solve_opts& o, cudaStream_t s) {
  const size_t bytes = (size_t)h->n * h->P * sizeof(double);
  if (F != h->fF) SG_TRY_CUDA(cudaMemcpyAsync(h->fF, F, bytes, cudaMemcpyDeviceToDevice, s));
  if (o.use_x0 && U != h->fx) SG_TRY_CUDA(cudaMemcpyAsync(h->fx, U, bytes, cudaMemcpyDeviceToDevice, s));
  SG_TRY_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int), s));
  SG_TRY_CUDA(cudaMemsetAsync(h->iacc, 0, 2 * sizeof(long long), s));
  return SG_OK;
}

// After the solve's work has completed: status and statistics.
int solve_collect(sg_problem* h, const sg_solve_opts& o, sg_solve_stats* st, double wall_ms) {
  OuterCtl ctl;
  SG_TRY_CUDA(cudaMemcpy(&ctl, h->octl, sizeof ctl, cudaMemcpyDeviceToHost));
  SG_TRY_CUDA(cudaMemcpy(h->osc_host, h->osc, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost));
  SG_TRY_CUDA(cudaMemcpy(h->status_host, h->status, sizeof(int), cudaMemcpyDeviceToHost));
  const int iters = ctl.it;
  const int status = *h->status_host;
  const double rel = h->osc_host[SC_REL];
  int result = SG_OK;
  if (status & ST_OUTER_BREAKDOWN) result = SG_ERR_BREAKDOWN;
  else if (status & ST_INNER_NOT_SPD) result = SG_ERR_NOT_SPD;
  else if (!(rel <= o.tol)) result = SG_ERR_NO_CONVERGENCE;
  if (st) {
    std::vector<double> a(std::max(iters, 1)), b(std::max(iters, 1)), res(iters + 1);
    long long iacc[2];
    SG_TRY_CUDA(cudaMemcpy(iacc, h->iacc, sizeof iacc, cudaMemcpyDeviceToHost));
    SG_TRY_CUDA(cudaMemcpy(res.data(), h->hist_res, (iters + 1) * sizeof(double), cudaMemcpyDeviceToHost));
    if (iters > 0) {
      SG_TRY_CUDA(cudaMemcpy(a.data(), h->hist_alpha, iters * sizeof(double), cudaMemcpyDeviceToHost));
      SG_TRY_CUDA(cudaMemcpy(b.data(), h->hist_beta, iters * sizeof(double), cudaMemcpyDeviceToHost));
    }
    st->status = result;
    st->iterations = iters;
    st->rel_res = rel;
    st->true_rel_res = o.check_true_residual ? h->osc_host[SC_TRUE] : -1.0;
    st->inner_iters_total = iacc[0];
    st->inner_iters_max = (int)iacc[1];
    st->n_hist = iters + 1;
    for (int i = 0; i <= iters && i <= SG_MAX_HIST; ++i) st->res_hist[i] = res[i];
    for (int i = 0; i < iters; ++i) {
      st->alpha[i] = a[i];
      st->beta[i] = i + 1 < iters ? b[i] : 0.0;
    }
    st->kappa_est = lanczos_kappa(a.data(), b.data(), iters);
    st->solve_ms = wall_ms;
  }
  if (result == SG_ERR_NO_CONVERGENCE) set_error("sg_solve: no convergence in %d iterations", iters);
  if (result == SG_ERR_BREAKDOWN) set_error("sg_solve: breakdown (p^T A p <= 0 or non-finite value)");
  if (result == SG_ERR_NOT_SPD) set_error("sg_solve: inner solve lost definiteness");
  return result;
}

// Host blocks of a solve: page-locked memory (cudaHostAlloc, cudaHostRegister)
// is read and written by k_copy64 through its device mapping, the SMs moving
// the data over the host link; other host memory goes through
// cudaMemcpyAsync. After the solve's kernels, the copy engine moved a 2.09 GB
// block in 130-147 ms where the SMs took 10-12 ms (the link's rate, about
// 210 GB/s), so the SMs do it.
int copy_host(sg_problem* h, const double* src, double* dst, size_t n, bool to_device, cudaStream_t s) {
  const void* host = to_device ? (const void*)src : (const void*)dst;
  cudaPointerAttributes at;
  const bool pinned = cudaPointerGetAttributes(&at, host) == cudaSuccess && at.type == cudaMemoryTypeHost &&
                      at.devicePointer;
  cudaGetLastError();
  if (pinned)
    return to_device ? launch_copy64((const double*)at.devicePointer, dst, (long long)n, h->num_sms, s)
                     : launch_copy64(src, (double*)at.devicePointer, (long long)n, h->num_sms, s);
  SG_TRY_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost,
                              s));
  return SG_OK;
}

// host: F and U are host blocks (copy_host), else device blocks
static int solve_impl(sg_problem* h, const double* F, double* U, const sg_solve_opts& o, sg_solve_stats* st,
                      cudaStream_t s, bool host = false) {
  const auto t0 = std::chrono::steady_clock::now();
  const size_t N = (size_t)h->n * h->P;
  SG_TRY(solve_prepare(h, o));
  if (host) {
    SG_TRY(copy_host(h, F, h->fF, N, true, s));
    if (o.use_x0) SG_TRY(copy_host(h, U, h->fx, N, true, s));
    SG_TRY(solve_stage_in(h, h->fF, h->fx, o, s));   // the device copies are in place: no-ops
  } else {
    SG_TRY(solve_stage_in(h, F, U, o, s));
  }
  SG_TRY(run_graph(h, solve_key(o), [&](cudaStream_t cs) {
    return o.schur_reduced ? enqueue_schur_solve(h, o, cs) : enqueue_solve(h, o, cs);
  }, s));
  if (host)
    SG_TRY(copy_host(h, o.schur_reduced ? h->fz : h->fx, U, N, false, s));
  else
    SG_TRY_CUDA(cudaMemcpyAsync(U, o.schur_reduced ? h->fz : h->fx, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  SG_TRY_CUDA(cudaStreamSynchronize(s));
  return solve_collect(h, o, st,
                       std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
}

}  // namespace sghsc

using namespace sghsc;

namespace sghsc {

int check_solve_opts(const sg_problem* h, const sg_solve_opts* opts) {
  if (!h || !opts || opts->maxit < 1 || !(opts->tol >= 0.0) ||
      (opts->precond != SG_PREC_NONE && opts->precond != SG_PREC_MEAN && opts->precond != SG_PREC_HSC &&
       opts->precond != SG_PREC_BGS)) {
    set_error("sg_solve: invalid options");
    return SG_ERR_INVALID_ARG;
  }
  if (opts->precond != SG_PREC_NONE || opts->schur_reduced) {
    if (opts->prec.precision != SG_F32 && opts->prec.precision != SG_F64) {
      set_error("sg_solve: invalid preconditioner precision");
      return SG_ERR_INVALID_ARG;
    }
    SG_TRY(check_prec_opts(opts->prec));
    SG_TRY(check_inner_support(h, opts->prec, "sg_solve"));
  }
  if (opts->schur_reduced && h->q >= 0) {
    set_error("sg_solve: the Schur-reduced system is built for the linear KL expansion only");
    return SG_ERR_UNSUPPORTED;
  }
  if (opts->schur_reduced && (h->p < 1 || opts->use_x0 || !(opts->schur_inner_tol >= 0.0))) {
    set_error("sg_solve: the Schur-reduced system needs p >= 1, use_x0 = 0 and schur_inner_tol >= 0");
    return SG_ERR_INVALID_ARG;
  }
  return SG_OK;
}

}  // namespace sghsc

extern "C" {

static int check_solve_call(sg_problem* h, const double* F, double* U, const sg_solve_opts* opts) {
  if (!h || !F || !U || !opts || F == U || opts->maxit < 1 || !(opts->tol >= 0.0) ||
      (opts->precond != SG_PREC_NONE && opts->precond != SG_PREC_MEAN && opts->precond != SG_PREC_HSC &&
       opts->precond != SG_PREC_BGS)) {
    set_error("sg_solve: invalid arguments");
    return SG_ERR_INVALID_ARG;
  }
  if (opts->precond != SG_PREC_NONE || opts->schur_reduced) {
    if (opts->prec.precision != SG_F32 && opts->prec.precision != SG_F64) {
      set_error("sg_solve: invalid preconditioner precision");
      return SG_ERR_INVALID_ARG;
    }
    SG_TRY(check_prec_opts(opts->prec));
    SG_TRY(check_inner_support(h, opts->prec, "sg_solve"));
  }
  if (opts->schur_reduced && h->q >= 0) {
    set_error("sg_solve: the Schur-reduced system is built for the linear KL expansion only");
    return SG_ERR_UNSUPPORTED;
  }
  if (opts->schur_reduced && (h->p < 1 || opts->use_x0 || !(opts->schur_inner_tol >= 0.0))) {
    set_error("sg_solve: the Schur-reduced system needs p >= 1, use_x0 = 0 and schur_inner_tol >= 0");
    return SG_ERR_INVALID_ARG;
  }
  return SG_OK;
}

int sg_solve(sg_problem* h, const double* F, double* U, const sg_solve_opts* opts, sg_solve_stats* stats,
             void* stream) {
  set_error("");
  SG_TRY(check_solve_call(h, F, U, opts));
  return solve_impl(h, F, U, *opts, stats, (cudaStream_t)stream);
}

int sg_solve_host(sg_problem* h, const double* F_host, double* U_host, const sg_solve_opts* opts,
                  sg_solve_stats* stats, void* stream) {
  set_error("");
  SG_TRY(check_solve_call(h, F_host, U_host, opts));
  return solve_impl(h, F_host, U_host, *opts, stats, (cudaStream_t)stream, true);
}

}  // extern "C"
