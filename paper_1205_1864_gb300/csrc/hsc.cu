// Algorithm 1 (Sec. 4): the hierarchical Schur complement preconditioner
// M_P : r_P -> u_P, and the mean-based preconditioner I (x) A_0^{-1} (Sec. 6).
//
// Storage reading of Algorithm 1: one working residual holds r_P; the
// pre-correction at level l overwrites its degree-(l-1) columns with
// g_{l-1} = r_l^{l-1} - B_l D_l^{-1} r_l^l (for the linear KL expansion B_l
// reaches degree l-1 only); the post-correction at level l uses the degree-l
// columns of that working residual. The D_l^{-1} actions are batched inner
// PCG solves on A_0 (all columns of one degree level in one batch); the loops
// over levels stay sequential, as Sec. 6 notes.
//
// Mixed precision (precision == SG_F32): the working residual, the inner
// solves and the level products run in FP32; with top_level_f64 the two
// level-p products read the FP64 input and accumulate in FP64.
//
// Everything here is enqueued inside a CUDA graph capture (the inner solves
// are device-controlled WHILE loops); the public entry points build the graph
// once per option set and replay it.
#include <cstdio>

#include "graph.cuh"
#include "sghsc_internal.cuh"
#include "vec.cuh"

namespace sghsc {

// Workspace of the nested D_l solves of the gPC case (before any capture).
static int ensure_level(sg_problem* h, const sg_prec_opts& o) {
  const int cap = std::min(o.level_maxit, 100000) + 2;
  if (h->lx && h->lhist_cap >= cap) return SG_OK;
  if (h->capturing) {
    set_error("level workspace must be allocated before graph capture");
    return SG_ERR_UNSUPPORTED;
  }
  if (h->lx) {
    clear_graphs(h);
    SG_TRY_CUDA(cudaDeviceSynchronize());
  }
  for (void* b : {(void*)h->lx, (void*)h->lr, (void*)h->lz, (void*)h->lp, (void*)h->lq, (void*)h->lb, (void*)h->lctl,
                  (void*)h->lsc, (void*)h->lhist_alpha, (void*)h->lhist_beta, (void*)h->lhist_res})
    cudaFree(b);
  // a failed allocation below leaves null pointers and no capacity, never a freed buffer
  h->lx = h->lr = h->lz = h->lp = h->lq = h->lb = nullptr;
  h->lctl = nullptr;
  h->lsc = h->lhist_alpha = h->lhist_beta = h->lhist_res = nullptr;
  h->lhist_cap = 0;
  const size_t bytes = (size_t)h->n * std::max(h->wmax, 1) * sizeof(double);
  for (double** b : {&h->lx, &h->lr, &h->lz, &h->lp, &h->lq, &h->lb}) SG_TRY_CUDA(cudaMalloc((void**)b, bytes));
  SG_TRY_CUDA(cudaMalloc((void**)&h->lctl, sizeof(OuterCtl)));
  SG_TRY_CUDA(cudaMemset(h->lctl, 0, sizeof(OuterCtl)));
  SG_TRY_CUDA(cudaMalloc((void**)&h->lsc, SC_COUNT * sizeof(double)));
  SG_TRY_CUDA(cudaMalloc((void**)&h->lhist_alpha, cap * sizeof(double)));
  SG_TRY_CUDA(cudaMalloc((void**)&h->lhist_beta, cap * sizeof(double)));
  SG_TRY_CUDA(cudaMalloc((void**)&h->lhist_res, cap * sizeof(double)));
  h->lhist_cap = cap;
  return SG_OK;
}

// D_l^{-1} of the gPC case (Sec. 6, lognormal: D_l = sum_i A_i (x) G_i[l, l]
// is not block diagonal, so "the solves involving D_l" are iterative): a
// flexible CG on the n x w_l level block with the operator D_l (the SG product
// restricted to the level, its i = 0 term the identity in chaos) and the
// mean-based preconditioner I (x) A_0^{-1} (the batched inner PCG on A_0,
// inner_tol), zero start, to level_tol. It reuses the outer iteration's
// kernels with its own control block and scalars, one nesting level deeper.
static int level_solve(sg_problem* h, int l, const double* src, int lds, double* dst, int ldd, const sg_prec_opts& o,
                       cudaStream_t s) {
  const int n = h->n, w = h->off[l + 1] - h->off[l];
  if (w <= 0) return SG_OK;
  const long long N = (long long)n * w;
  const int vg = std::min(vec_grid(N), h->opart_blocks);
  OuterArgs a0;
  a0.part = h->opart;
  a0.ctl = h->lctl;
  a0.sc = h->lsc;
  a0.hist_alpha = h->lhist_alpha;
  a0.hist_beta = h->lhist_beta;
  a0.hist_res = h->lhist_res;
  a0.status = h->status;
  a0.flexible = 1;
  a0.maxit = std::min(o.level_maxit, h->lhist_cap - 2);
  a0.tol = o.level_tol;
  a0.cond = 0;
  a0.has_cond = 0;
  a0.flag = nullptr;
  auto with = [&](const LoopCtl& lc) {
    OuterArgs a = a0;
    a.cond = lc.cond;
    a.has_cond = lc.has_cond;
    a.flag = lc.flag;
    return a;
  };
  SG_TRY(launch_cast(src, SG_F64, lds, h->lb, SG_F64, w, n, w, s));
  auto pre = [&](cudaStream_t ps, const LoopCtl& lc) -> int {
    const OuterArgs a = with(lc);
    SG_TRY_CUDA(cudaMemsetAsync(h->lx, 0, N * sizeof(double), ps));
    { k_outer_init<<<vg, 256, 0, ps>>>(N, h->lb, nullptr, h->lr, a); ::sghsc::note_launch(); }
    SG_CHECK_LAUNCH();
    return SG_OK;
  };
  auto body = [&](cudaStream_t bs, const LoopCtl& lc) -> int {
    const OuterArgs a = with(lc);
    SG_TRY(inner_solve(h, SG_F64, h->lr, w, SG_F64, h->lz, w, SG_F64, w, o, bs));
    { k_outer_dots<<<vg, 256, 0, bs>>>(N, h->lz, h->lr, h->lq, a); ::sghsc::note_launch(); }
    { k_schur_p<<<vg, 256, 0, bs>>>(N, h->lz, h->lp, a); ::sghsc::note_launch(); }
    SG_TRY(launch_block_matvec(h, SG_F64, SG_F64, SG_F64, SG_F64, h->lp, w, w, h->dlev[l], true, nullptr, 0, 1.0, 0.0,
                               h->lq, w, bs));
    { k_schur_pq<<<vg, 256, 0, bs>>>(N, h->lp, h->lq, a); ::sghsc::note_launch(); }
    { k_outer_update<<<vg, 256, 0, bs>>>(N, h->lp, h->lp, h->lq, h->lx, h->lr, a); ::sghsc::note_launch(); }
    SG_CHECK_LAUNCH();
    return SG_OK;
  };
  SG_TRY(capture_while(h, s, pre, body));
  return launch_cast(h->lx, SG_F64, w, dst, SG_F64, ldd, n, w, s);
}

// D_l^{-1}: the batched inner PCG on A_0 (linear KL expansion, Lemma of Sec. 3)
// or the nested level CG (gPC coefficient).
static int dsolve64(sg_problem* h, int l, const double* src, int lds, double* dst, int ldd, const sg_prec_opts& o,
                    cudaStream_t s) {
  if (h->q >= 0 && l >= 1) return level_solve(h, l, src, lds, dst, ldd, o, s);
  return inner_solve(h, SG_F64, src, lds, SG_F64, dst, ldd, SG_F64, h->off[l + 1] - h->off[l], o, s);
}

static int ensure_hsc32(sg_problem* h) {
  if (h->R32) return SG_OK;
  const size_t np = (size_t)h->n * h->P;
  SG_TRY_CUDA(cudaMalloc((void**)&h->R32, np * sizeof(float)));
  SG_TRY_CUDA(cudaMalloc((void**)&h->Z32, np * sizeof(float)));
  SG_TRY_CUDA(cudaMalloc((void**)&h->T32, (size_t)h->n * std::max(h->wmax, 1) * sizeof(float)));
  return SG_OK;
}

static int ensure_hsc64(sg_problem* h) {
  if (h->R64w) return SG_OK;
  const size_t np = (size_t)h->n * h->P;
  SG_TRY_CUDA(cudaMalloc((void**)&h->R64w, np * sizeof(double)));
  SG_TRY_CUDA(cudaMalloc((void**)&h->T64, (size_t)h->n * std::max(h->wmax, 1) * sizeof(double)));
  return SG_OK;
}

// Allocate everything a preconditioner application needs (before any capture).
int prepare_precond(sg_problem* h, int kind, const sg_prec_opts& o) {
  SG_TRY(check_prec_opts(o));
  const int dt = o.precision == SG_F32 ? SG_F32 : SG_F64;
  if (h->q >= 0 && (kind == SG_PREC_BGS || (kind == SG_PREC_HSC && dt == SG_F32))) {
    set_error("gPC coefficient: Algorithm 1 runs in FP64 (nested D_l solves); block Gauss-Seidel is not built");
    return SG_ERR_UNSUPPORTED;
  }
  if (h->q >= 0 && kind == SG_PREC_HSC && o.md_m0) {
    set_error("gPC coefficient: D_l is not I (x) A_0, so M_0 cannot stand in for D_l^{-1} (md_m0)");
    return SG_ERR_UNSUPPORTED;
  }
  if (h->q >= 0 && kind == SG_PREC_HSC) SG_TRY(ensure_level(h, o));
  if (kind == SG_PREC_HSC || kind == SG_PREC_BGS) {
    SG_TRY(ensure_inner_work(h, dt, h->wmax));
    SG_TRY(dt == SG_F32 ? ensure_hsc32(h) : ensure_hsc64(h));
  } else if (kind == SG_PREC_MEAN) {
    SG_TRY(ensure_inner_work(h, dt, std::max(std::min(h->P, 1024), h->wmax)));
  }
  return SG_OK;
}

// Algorithm 1 on the hierarchy of levels 0..p of blocks with leading
// dimension P (p = h->p, P = h->P for the full system; p - 1 and the width of
// levels 0..p-1 for the Schur-reduced one).
int hsc_apply_lv(sg_problem* h, const double* R, double* Z, const sg_prec_opts& o, cudaStream_t s, int p, int P) {
  const int n = h->n;
  const std::vector<int>& off = h->off;
  if (o.precision == SG_F32) {
    float* R32 = h->R32;
    float* Z32 = h->Z32;
    const bool top64 = o.top_level_f64 != 0;
    const int acc64 = o.df64 ? ACC_DF64 : SG_F64;   // FP64-accurate accumulation: FP64 or double-float
    // With the FP64 top level only levels 0..p-2 of R are needed in FP32 (the
    // pre-correction at level l reads level l-1 in place): the degree-p solve
    // gathers its columns from R (converting on the way), and the top-level
    // pre-correction writes level p-1 from R itself.
    const bool m0_pre = (o.md_m0 & 1) != 0, m0_post = (o.md_m0 & 2) != 0;   // eq. (general-prec) variants
    const bool cast_all = !(top64 && p >= 1) || m0_pre;
    const int cast_cols = cast_all ? P : off[std::max(p - 1, 0)];
    if (cast_cols > 0) SG_TRY(launch_cast(R, SG_F64, P, R32, SG_F32, P, n, cast_cols, s));
    // first loop, l = p..1: D_l^{-1} on the degree-l columns, then the pre-correction
    for (int l = p; l >= 1; --l) {
      const int lo = off[l], w = off[l + 1] - off[l], lo1 = off[l - 1];
      if (m0_pre)
        SG_TRY(m0_apply(h, SG_F32, R32 + lo, P, Z32 + lo, P, w, o, s));
      else if (l == p && !cast_all)
        SG_TRY(inner_solve(h, SG_F32, R + lo, P, SG_F64, Z32 + lo, P, SG_F32, w, o, s));
      else
        SG_TRY(inner_solve(h, SG_F32, R32 + lo, P, SG_F32, Z32 + lo, P, SG_F32, w, o, s));
      if (l == p && top64)
        SG_TRY(launch_block_matvec(h, SG_F32, acc64, SG_F64, SG_F32, Z32 + lo, P, w, h->pre[l], false, R + lo1, P,
                                   -1.0, 1.0, R32 + lo1, P, s));
      else
        SG_TRY(launch_block_matvec(h, SG_F32, SG_F32, SG_F32, SG_F32, Z32 + lo, P, w, h->pre[l], false, R32 + lo1, P,
                                   -1.0, 1.0, R32 + lo1, P, s));
    }
    // mean-value problem A_0 u_0 = g_0
    SG_TRY(inner_solve(h, SG_F32, R32, P, SG_F32, Z32, P, SG_F32, off[1] - off[0], o, s));
    // second loop, l = 1..p: post-correction, then D_l^{-1}
    for (int l = 1; l <= p; ++l) {
      const int lo = off[l], w = off[l + 1] - off[l], lo1 = off[l - 1], w1 = off[l] - off[l - 1];
      if (l == p && top64)
        SG_TRY(launch_block_matvec(h, SG_F32, acc64, SG_F64, SG_F32, Z32 + lo1, P, w1, h->post[l], false, R + lo, P,
                                   -1.0, 1.0, h->T32, w, s));
      else
        SG_TRY(launch_block_matvec(h, SG_F32, SG_F32, SG_F32, SG_F32, Z32 + lo1, P, w1, h->post[l], false, R32 + lo,
                                   P, -1.0, 1.0, h->T32, w, s));
      if (m0_post)
        SG_TRY(m0_apply(h, SG_F32, h->T32, w, Z32 + lo, P, w, o, s));
      else
        SG_TRY(inner_solve(h, SG_F32, h->T32, w, SG_F32, Z32 + lo, P, SG_F32, w, o, s));
    }
    if (Z) SG_TRY(launch_cast(Z32, SG_F32, P, Z, SG_F64, P, n, P, s));   // Z null: z stays in Z32
    return SG_OK;
  }
  // all FP64 (the pre-correction product writes the lower levels it reaches:
  // level l-1 for the linear KL expansion, every lower level for a gPC one)
  double* Rw = h->R64w;
  SG_TRY_CUDA(cudaMemcpyAsync(Rw, R, (size_t)n * P * sizeof(double), cudaMemcpyDeviceToDevice, s));
  for (int l = p; l >= 1; --l) {
    const int lo = off[l], w = off[l + 1] - off[l];
    const EdgeList& B = h->pre[l];
    if (o.md_m0 & 1)
      SG_TRY(m0_apply(h, SG_F64, Rw + lo, P, Z + lo, P, w, o, s));
    else
      SG_TRY(dsolve64(h, l, Rw + lo, P, Z + lo, P, o, s));
    SG_TRY(launch_block_matvec(h, SG_F64, SG_F64, SG_F64, SG_F64, Z + lo, P, w, B, false, Rw + B.out0, P, -1.0,
                               1.0, Rw + B.out0, P, s));
  }
  SG_TRY(dsolve64(h, 0, Rw, P, Z, P, o, s));
  for (int l = 1; l <= p; ++l) {
    const int lo = off[l], w = off[l + 1] - off[l];
    const EdgeList& C = h->post[l];
    SG_TRY(launch_block_matvec(h, SG_F64, SG_F64, SG_F64, SG_F64, Z + C.in0, P, C.nin, C, false, Rw + lo, P, -1.0,
                               1.0, h->T64, w, s));
    if (o.md_m0 & 2)
      SG_TRY(m0_apply(h, SG_F64, h->T64, w, Z + lo, P, w, o, s));
    else
      SG_TRY(dsolve64(h, l, h->T64, w, Z + lo, P, o, s));
  }
  return SG_OK;
}

// Block symmetric Gauss-Seidel with zero initial guess (M_bGS, Sec. 6): a
// forward sweep over the chaos blocks in graded order, then a backward one.
// With the linear KL expansion a block of degree d couples only to degrees
// d - 1 and d + 1 (the blocks of one degree do not couple), so the sweep over
// chaos indices is a sweep over degree levels with all w_d solves of a level
// in one batch:
//   forward   T_d = R_d - C_d Z_{d-1},  Z_d = A_0^{-1} T_d          d = 0..p
//   backward  Z_d = A_0^{-1} (T_d - B_{d+1} Z_{d+1})                d = p-1..0
// (the backward step at d = p would repeat the forward one exactly). T_d is
// kept from the forward sweep in the working residual (in place of R_d,
// which is not needed again), so the C_d products are not recomputed: n_m
// block products instead of the 1.5 n_m the paper counts, the same result.
// Mixed precision as in Algorithm 1; with top_level_f64 the level-p forward
// product reads the FP64 input and accumulates in FP64.
int bgs_apply_lv(sg_problem* h, const double* R, double* Z, const sg_prec_opts& o, cudaStream_t s, int p, int P) {
  const int n = h->n;
  const std::vector<int>& off = h->off;
  if (o.precision == SG_F32) {
    float* R32 = h->R32;
    float* Z32 = h->Z32;
    const bool top64 = o.top_level_f64 != 0;
    SG_TRY(launch_cast(R, SG_F64, P, R32, SG_F32, P, n, P, s));
    SG_TRY(inner_solve(h, SG_F32, R32, P, SG_F32, Z32, P, SG_F32, off[1] - off[0], o, s));
    for (int d = 1; d <= p; ++d) {
      const int lo = off[d], w = off[d + 1] - off[d], lo1 = off[d - 1], w1 = off[d] - off[d - 1];
      if (d == p && top64)
        SG_TRY(launch_block_matvec(h, SG_F32, o.df64 ? ACC_DF64 : SG_F64, SG_F64, SG_F32, Z32 + lo1, P, w1,
                                   h->post[d], false, R + lo, P, -1.0, 1.0, R32 + lo, P, s));
      else
        SG_TRY(launch_block_matvec(h, SG_F32, SG_F32, SG_F32, SG_F32, Z32 + lo1, P, w1, h->post[d], false, R32 + lo,
                                   P, -1.0, 1.0, R32 + lo, P, s));
      SG_TRY(inner_solve(h, SG_F32, R32 + lo, P, SG_F32, Z32 + lo, P, SG_F32, w, o, s));
    }
    for (int d = p - 1; d >= 0; --d) {
      const int lo = off[d], w = off[d + 1] - off[d], lo2 = off[d + 1], w2 = off[d + 2] - off[d + 1];
      SG_TRY(launch_block_matvec(h, SG_F32, SG_F32, SG_F32, SG_F32, Z32 + lo2, P, w2, h->pre[d + 1], false, R32 + lo, P,
                                 -1.0, 1.0, R32 + lo, P, s));
      SG_TRY(inner_solve(h, SG_F32, R32 + lo, P, SG_F32, Z32 + lo, P, SG_F32, w, o, s));
    }
    if (Z) SG_TRY(launch_cast(Z32, SG_F32, P, Z, SG_F64, P, n, P, s));   // Z null: z stays in Z32
    return SG_OK;
  }
  double* Rw = h->R64w;
  SG_TRY_CUDA(cudaMemcpyAsync(Rw, R, (size_t)n * P * sizeof(double), cudaMemcpyDeviceToDevice, s));
  SG_TRY(inner_solve(h, SG_F64, Rw, P, SG_F64, Z, P, SG_F64, off[1] - off[0], o, s));
  for (int d = 1; d <= p; ++d) {
    const int lo = off[d], w = off[d + 1] - off[d], lo1 = off[d - 1], w1 = off[d] - off[d - 1];
    SG_TRY(launch_block_matvec(h, SG_F64, SG_F64, SG_F64, SG_F64, Z + lo1, P, w1, h->post[d], false, Rw + lo, P, -1.0,
                               1.0, Rw + lo, P, s));
    SG_TRY(inner_solve(h, SG_F64, Rw + lo, P, SG_F64, Z + lo, P, SG_F64, w, o, s));
  }
  for (int d = p - 1; d >= 0; --d) {
    const int lo = off[d], w = off[d + 1] - off[d], lo2 = off[d + 1], w2 = off[d + 2] - off[d + 1];
    SG_TRY(launch_block_matvec(h, SG_F64, SG_F64, SG_F64, SG_F64, Z + lo2, P, w2, h->pre[d + 1], false, Rw + lo, P,
                               -1.0, 1.0, Rw + lo, P, s));
    SG_TRY(inner_solve(h, SG_F64, Rw + lo, P, SG_F64, Z + lo, P, SG_F64, w, o, s));
  }
  return SG_OK;
}

int hsc_apply_impl(sg_problem* h, const double* R, double* Z, const sg_prec_opts& o, cudaStream_t s) {
  return hsc_apply_lv(h, R, Z, o, s, h->p, h->P);
}

int bgs_apply_impl(sg_problem* h, const double* R, double* Z, const sg_prec_opts& o, cudaStream_t s) {
  return bgs_apply_lv(h, R, Z, o, s, h->p, h->P);
}

// I (x) A_0^{-1} on the P columns of a block with leading dimension P.
int mean_apply_lv(sg_problem* h, const double* R, double* Z, const sg_prec_opts& o, cudaStream_t s, int P) {
  const int chunk = std::min(P, 1024);
  const int dt = o.precision == SG_F32 ? SG_F32 : SG_F64;
  for (int c0 = 0; c0 < P; c0 += chunk) {
    const int w = std::min(chunk, P - c0);
    SG_TRY(inner_solve(h, dt, R + c0, P, SG_F64, Z + c0, P, SG_F64, w, o, s));
  }
  return SG_OK;
}

int mean_apply_impl(sg_problem* h, const double* R, double* Z, const sg_prec_opts& o, cudaStream_t s) {
  return mean_apply_lv(h, R, Z, o, s, h->P);
}

static int check_prec_call(sg_problem* h, const void* R, const void* Z, const sg_prec_opts* o, const char* name) {
  if (!h || !R || !Z || !o || R == Z || (o->precision != SG_F32 && o->precision != SG_F64)) {
    set_error("%s: invalid arguments", name);
    return SG_ERR_INVALID_ARG;
  }
  SG_TRY(check_prec_opts(*o));
  return check_inner_support(h, *o, name);
}

static int finish_status(sg_problem* h, cudaStream_t s) {
  SG_TRY_CUDA(cudaMemcpyAsync(h->status_host, h->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  SG_TRY_CUDA(cudaStreamSynchronize(s));
  if (*h->status_host & ST_INNER_NOT_SPD) {
    set_error("inner solve lost definiteness (p^T A_0 p <= 0 or non-finite residual)");
    return SG_ERR_NOT_SPD;
  }
  return SG_OK;
}

// Graph-run preconditioner application: R is staged into the outer residual
// buffer, the result comes back from the outer preconditioned-residual buffer.
static int precond_entry(sg_problem* h, int kind, const double* R, double* Z, const sg_prec_opts& o,
                         cudaStream_t s) {
  SG_TRY(ensure_outer(h));
  SG_TRY(prepare_precond(h, kind, o));
  const size_t bytes = (size_t)h->n * h->P * sizeof(double);
  SG_TRY_CUDA(cudaMemcpyAsync(h->fr, R, bytes, cudaMemcpyDeviceToDevice, s));
  SG_TRY_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int), s));
  const std::string key = std::string(kind == SG_PREC_HSC ? "hsc|" : kind == SG_PREC_BGS ? "bgs|" : "mean|") +
                          opts_key(o);
  SG_TRY(run_graph(h, key, [&](cudaStream_t cs) {
    if (kind == SG_PREC_HSC) return hsc_apply_impl(h, h->fr, h->fz, o, cs);
    if (kind == SG_PREC_BGS) return bgs_apply_impl(h, h->fr, h->fz, o, cs);
    return mean_apply_impl(h, h->fr, h->fz, o, cs);
  }, s));
  SG_TRY_CUDA(cudaMemcpyAsync(Z, h->fz, bytes, cudaMemcpyDeviceToDevice, s));
  return finish_status(h, s);
}

}  // namespace sghsc

using namespace sghsc;

extern "C" {

int hsc_precond_apply(sg_problem* h, const double* R, double* Z, const sg_prec_opts* opts, void* stream) {
  set_error("");
  SG_TRY(check_prec_call(h, R, Z, opts, "hsc_precond_apply"));
  return precond_entry(h, SG_PREC_HSC, R, Z, *opts, (cudaStream_t)stream);
}

int bgs_precond_apply(sg_problem* h, const double* R, double* Z, const sg_prec_opts* opts, void* stream) {
  set_error("");
  SG_TRY(check_prec_call(h, R, Z, opts, "bgs_precond_apply"));
  return precond_entry(h, SG_PREC_BGS, R, Z, *opts, (cudaStream_t)stream);
}

int mean_precond_apply(sg_problem* h, const double* R, double* Z, const sg_prec_opts* opts, void* stream) {
  set_error("");
  SG_TRY(check_prec_call(h, R, Z, opts, "mean_precond_apply"));
  return precond_entry(h, SG_PREC_MEAN, R, Z, *opts, (cudaStream_t)stream);
}

int sg_vcycle_apply(sg_problem* h, const void* B, void* X, int w, int dtype, const sg_prec_opts* opts,
                    void* stream) {
  set_error("");
  if (!h || !B || !X || !opts || w <= 0 || w > 1024 || (dtype != SG_F64 && dtype != SG_F32)) {
    set_error("sg_vcycle_apply: invalid arguments");
    return SG_ERR_INVALID_ARG;
  }
  sg_prec_opts o = *opts;
  o.m0 = SG_M0_VCYCLE;   // this entry point is the V-cycle itself
  SG_TRY(check_inner_support(h, o, "sg_vcycle_apply"));
  return inner_vcycle(h, dtype, B, X, w, o, (cudaStream_t)stream);
}

int sg_inner_solve(sg_problem* h, const void* B, void* X, int w, int dtype, const sg_prec_opts* opts, int* iters,
                   void* stream) {
  set_error("");
  if (!h || !B || !X || !opts || w <= 0 || w > 1024 || (dtype != SG_F64 && dtype != SG_F32)) {
    set_error("sg_inner_solve: invalid arguments");
    return SG_ERR_INVALID_ARG;
  }
  SG_TRY(check_prec_opts(*opts));
  SG_TRY(check_inner_support(h, *opts, "sg_inner_solve"));
  cudaStream_t s = (cudaStream_t)stream;
  SG_TRY(ensure_inner_work(h, dtype, std::max(w, h->wmax)));
  const size_t es = dtype == SG_F64 ? 8 : 4;
  const size_t bytes = (size_t)h->n * w * es;
  if (h->io_bytes < bytes) {
    clear_graphs(h);
    SG_TRY_CUDA(cudaDeviceSynchronize());
    cudaFree(h->io_in);
    cudaFree(h->io_out);
    h->io_in = h->io_out = nullptr;
    h->io_bytes = 0;
    SG_TRY_CUDA(cudaMalloc(&h->io_in, bytes));
    SG_TRY_CUDA(cudaMalloc(&h->io_out, bytes));
    h->io_bytes = bytes;
  }
  SG_TRY_CUDA(cudaMemcpyAsync(h->io_in, B, bytes, cudaMemcpyDeviceToDevice, s));
  SG_TRY_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int), s));
  char key[320];
  snprintf(key, sizeof key, "inner|d%d|w%d|%s", dtype, w, opts_key(*opts).c_str());
  const sg_prec_opts o = *opts;
  SG_TRY(run_graph(h, key, [&](cudaStream_t cs) {
    return inner_solve(h, dtype, h->io_in, w, dtype, h->io_out, w, dtype, w, o, cs);
  }, s));
  SG_TRY_CUDA(cudaMemcpyAsync(X, h->io_out, bytes, cudaMemcpyDeviceToDevice, s));
  if (iters) {
    const InnerWork& iw = dtype == SG_F64 ? h->iw64 : h->iw32;
    SG_TRY_CUDA(cudaMemcpyAsync(iters, iw.iters, sizeof(int) * w, cudaMemcpyDeviceToHost, s));
  }
  return finish_status(h, s);
}

}  // extern "C"
