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
    h->opart_blocks = need;
    SG_TRY_CUDA(cudaMalloc((void**)&h->opart, (size_t)h->opart_blocks * 2 * sizeof(double)));
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
    SG_TRY(precond(h, o.precond, h->fr, h->fz, o.prec, bs));
    { k_outer_dots<<<vg, 256, 0, bs>>>(N, h->fz, h->fr, h->fq, a); ::sghsc::note_launch(); }
    SG_TRY(launch_outer_matvec(h, a, bs));
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

std::string opts_key(const sg_prec_opts& o) {
  char buf[256];
  snprintf(buf, sizeof buf, "p%d|t%d|tol%.17g|mi%d|fx%d|nu%d|om%.17g|m%d", o.precision, o.top_level_f64,
           o.inner_tol, o.inner_maxit, o.inner_fixed_iters, o.nu, o.omega, o.m0);
  return buf;
}

int solve_prepare(sg_problem* h, const sg_solve_opts& o) {
  SG_TRY(ensure_outer(h));
  if (o.precond != SG_PREC_NONE) SG_TRY(prepare_precond(h, o.precond, o.prec));
  return SG_OK;
}

std::string solve_key(const sg_solve_opts& o) {
  char key[512];
  snprintf(key, sizeof key, "solve|k%d|%s|tol%.17g|mi%d|fl%d|x0%d|tr%d", o.precond,
           o.precond == SG_PREC_NONE ? "-" : opts_key(o.prec).c_str(), o.tol, o.maxit, o.flexible, o.use_x0,
           o.check_true_residual);
  return key;
}

// Copy the right-hand side (and the initial guess) into the handle's buffers.
int solve_stage_in(sg_problem* h, const double* F, const double* U, const sg_solve_opts& o, cudaStream_t s) {
  const size_t bytes = (size_t)h->n * h->P * sizeof(double);
  SG_TRY_CUDA(cudaMemcpyAsync(h->fF, F, bytes, cudaMemcpyDeviceToDevice, s));
  if (o.use_x0) SG_TRY_CUDA(cudaMemcpyAsync(h->fx, U, bytes, cudaMemcpyDeviceToDevice, s));
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

static int solve_impl(sg_problem* h, const double* F, double* U, const sg_solve_opts& o, sg_solve_stats* st,
                      cudaStream_t s) {
  const auto t0 = std::chrono::steady_clock::now();
  SG_TRY(solve_prepare(h, o));
  SG_TRY(solve_stage_in(h, F, U, o, s));
  SG_TRY(run_graph(h, solve_key(o), [&](cudaStream_t cs) { return enqueue_solve(h, o, cs); }, s));
  SG_TRY_CUDA(cudaMemcpyAsync(U, h->fx, (size_t)h->n * h->P * sizeof(double), cudaMemcpyDeviceToDevice, s));
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
  if (opts->precond != SG_PREC_NONE) {
    if (opts->prec.precision != SG_F32 && opts->prec.precision != SG_F64) {
      set_error("sg_solve: invalid preconditioner precision");
      return SG_ERR_INVALID_ARG;
    }
    SG_TRY(check_prec_opts(opts->prec));
    SG_TRY(check_inner_support(h, opts->prec, "sg_solve"));
  }
  return SG_OK;
}

}  // namespace sghsc

extern "C" {

int sg_solve(sg_problem* h, const double* F, double* U, const sg_solve_opts* opts, sg_solve_stats* stats,
             void* stream) {
  set_error("");
  if (!h || !F || !U || !opts || F == U || opts->maxit < 1 || !(opts->tol >= 0.0) ||
      (opts->precond != SG_PREC_NONE && opts->precond != SG_PREC_MEAN && opts->precond != SG_PREC_HSC &&
       opts->precond != SG_PREC_BGS)) {
    set_error("sg_solve: invalid arguments");
    return SG_ERR_INVALID_ARG;
  }
  if (opts->precond != SG_PREC_NONE) {
    if (opts->prec.precision != SG_F32 && opts->prec.precision != SG_F64) {
      set_error("sg_solve: invalid preconditioner precision");
      return SG_ERR_INVALID_ARG;
    }
    SG_TRY(check_prec_opts(opts->prec));
    SG_TRY(check_inner_support(h, opts->prec, "sg_solve"));
  }
  return solve_impl(h, F, U, *opts, stats, (cudaStream_t)stream);
}

}  // extern "C"
