// K6: many independent SG systems (uneven mesh size, M and p) solved by one
// graph launch, and the autotuner that picks the block shape of the SG product
// per problem.
//
// The batch graph has one branch per system: each branch is that system's
// whole solve (outer flexible CG with its nested device-controlled inner
// loops, graph.cu / fcg.cu), captured on its own stream between a fork and a
// join event. One cudaGraphLaunch then runs every system; the branches are
// independent, so the GPU schedules their kernels side by side and the small
// systems fill the gaps of the large ones. Nothing returns to the host until
// all systems are done.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "graph.cuh"
#include "sghsc_internal.cuh"
#include "vec.cuh"

struct sg_batch {
  std::vector<sg_problem*> hs;
  std::vector<long long> gens;   // workspace generation of each handle when the graphs were built
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaStream_t cs = nullptr;
  std::map<std::string, sghsc::GraphEntry> graphs;
};

namespace sghsc {

static void batch_clear(sg_batch* b) {
  for (auto& kv : b->graphs) {
    cudaGraphExecDestroy(kv.second.exec);
    cudaGraphDestroy(kv.second.graph);
  }
  b->graphs.clear();
}

static int batch_build(sg_batch* b, const sg_solve_opts& o, cudaGraph_t* out) {
  SG_TRY_CUDA(cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeRelaxed));
  int r = SG_OK;
  cudaError_t e = cudaEventRecord(b->fork, b->cs);
  for (size_t i = 0; i < b->hs.size() && r == SG_OK && e == cudaSuccess; ++i) {
    sg_problem* h = b->hs[i];
    e = cudaStreamWaitEvent(b->branch[i], b->fork, 0);
    if (e != cudaSuccess) break;
    h->capturing = true;
    h->cap_depth = 0;
    r = enqueue_solve(h, o, b->branch[i]);
    h->capturing = false;
    if (r != SG_OK) break;
    e = cudaEventRecord(b->join[i], b->branch[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cs, b->join[i], 0);
  }
  cudaGraph_t g = nullptr;
  cudaError_t ee = cudaStreamEndCapture(b->cs, &g);
  if (r != SG_OK || e != cudaSuccess || ee != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    if (r != SG_OK) return r;
    SG_TRY_CUDA(e != cudaSuccess ? e : ee);
  }
  *out = g;
  return SG_OK;
}

// host: F[i], U[i] are host blocks (copy_host), else device blocks
static int batch_solve(sg_batch* b, const double* const* F, double* const* U, const sg_solve_opts& o,
                       sg_solve_stats* stats, cudaStream_t s, bool host = false) {
  const auto t0 = std::chrono::steady_clock::now();
  for (sg_problem* h : b->hs) {
    SG_TRY(check_solve_opts(h, &o));
    SG_TRY(solve_prepare(h, o));
  }
  for (size_t i = 0; i < b->hs.size(); ++i) {
    sg_problem* h = b->hs[i];
    if (host) {
      const size_t N = (size_t)h->n * h->P;
      SG_TRY(copy_host(h, F[i], h->fF, N, true, s));
      if (o.use_x0) SG_TRY(copy_host(h, U[i], h->fx, N, true, s));
      SG_TRY(solve_stage_in(h, h->fF, h->fx, o, s));
    } else {
      SG_TRY(solve_stage_in(h, F[i], U[i], o, s));
    }
  }
  // a workspace reallocation in any handle invalidates the captured graphs
  bool stale = b->gens.size() != b->hs.size();
  for (size_t i = 0; !stale && i < b->hs.size(); ++i) stale = b->gens[i] != b->hs[i]->ws_gen;
  if (stale) {
    batch_clear(b);
    b->gens.clear();
    for (sg_problem* h : b->hs) b->gens.push_back(h->ws_gen);
  }
  const std::string key = solve_key(o);
  auto it = b->graphs.find(key);
  if (it == b->graphs.end()) {
    cudaGraph_t g = nullptr;
    SG_TRY(batch_build(b, o, &g));
    cudaGraphExec_t ex;
    cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
    if (ei != cudaSuccess) {
      cudaGraphDestroy(g);
      SG_TRY_CUDA(ei);
    }
    it = b->graphs.emplace(key, GraphEntry{g, ex}).first;
  }
  { SG_TRY_CUDA(cudaGraphLaunch(it->second.exec, s)); }
  for (size_t i = 0; i < b->hs.size(); ++i) {
    sg_problem* h = b->hs[i];
    if (host)
      SG_TRY(copy_host(h, h->fx, U[i], (size_t)h->n * h->P, false, s));
    else
      SG_TRY_CUDA(cudaMemcpyAsync(U[i], h->fx, (size_t)h->n * h->P * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  SG_TRY_CUDA(cudaStreamSynchronize(s));
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  int result = SG_OK;
  for (size_t i = 0; i < b->hs.size(); ++i) {
    const int r = solve_collect(b->hs[i], o, stats ? &stats[i] : nullptr, ms);
    if (r != SG_OK && result == SG_OK) result = r;
  }
  if (result != SG_OK) set_error("sg_batch_solve: at least one system did not converge or broke down (see stats)");
  return result;
}

// ---------------------------------------------------------------- autotune ---

// Candidate block sizes of the full product: powers of two from 64 to 1024 and
// the whole-warp sizes that give every thread 1, 2 or 4 outputs with at most
// 31 idle lanes (224 for P = 210).
static std::vector<int> block_candidates(int P) {
  std::vector<int> c = {64, 128, 256, 512, 1024};
  for (int m : {1, 2, 4}) {
    const int t = 32 * ceil_div(P, 32 * m);
    if (t >= 64 && t <= 1024 && std::find(c.begin(), c.end(), t) == c.end()) c.push_back(t);
  }
  return c;
}

// Time the full SG product with each candidate block size, in pair and in
// gather form, and keep the fastest.
static int autotune_k1(sg_problem* h, int dtype, cudaStream_t s) {
  const size_t es = dtype == SG_F64 ? 8 : 4;
  const size_t bytes = (size_t)h->n * h->P * es;
  void *X = nullptr, *Y = nullptr;
  SG_TRY_CUDA(cudaMalloc(&X, bytes));
  cudaError_t e = cudaMalloc(&Y, bytes);
  if (e != cudaSuccess) {
    cudaFree(X);
    SG_TRY_CUDA(e);
  }
  cudaMemsetAsync(X, 0, bytes, s);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const std::vector<int> cands = block_candidates(h->P);
  const int nc = (int)cands.size();
  int best = 0, best_pairs = 1;
  float best_ms = 1e30f;
  int r = SG_OK;
  for (int cand = 0; cand < 2 * nc && r == SG_OK; ++cand) {
    const int c = cands[cand % nc], pairs = cand < nc ? 1 : 0;
    if ((h->P + c - 1) / c > 8) continue;   // at most 8 outputs per thread
    if (pairs && h->q >= 0) continue;       // gPC: gather form only
    h->k1_threads[dtype] = c;
    h->k1_pairs[dtype] = pairs;
    r = launch_block_matvec(h, dtype, dtype, dtype, dtype, X, h->P, h->P, h->all, true, nullptr, 0, 1.0, 0.0, Y,
                            h->P, s);
    if (r != SG_OK) break;
    cudaEventRecord(e0, s);
    for (int rep = 0; rep < 5 && r == SG_OK; ++rep)
      r = launch_block_matvec(h, dtype, dtype, dtype, dtype, X, h->P, h->P, h->all, true, nullptr, 0, 1.0, 0.0, Y,
                              h->P, s);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r == SG_OK && ms < best_ms) {
      best_ms = ms;
      best = c;
      best_pairs = pairs;
    }
  }
  h->k1_threads[dtype] = best;
  h->k1_pairs[dtype] = h->q >= 0 ? 0 : best_pairs;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(X);
  cudaFree(Y);
  return r;
}

// Time the fused outer product (K1 with the CG update and p . q) with each
// candidate block size, in pair and in gather form, on the handle's own outer
// buffers and keep the fastest, for the FP64 product and separately for its
// double-float variant (df). It runs on whatever the buffers hold; every solve
// stages its right-hand side and resets the outer state before it starts.
static int autotune_outer(sg_problem* h, cudaStream_t s, bool df) {
  SG_TRY(ensure_outer(h));
  sg_solve_opts o;
  sg_default_solve_opts(&o);
  const OuterArgs a = outer_args(h, o);
  int& t_out = df ? h->outer_threads_df : h->outer_threads;
  int& p_out = df ? h->outer_pairs_df : h->outer_pairs;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const std::vector<int> cands = block_candidates(h->P);
  const int nc = (int)cands.size();
  int best = 0, best_pairs = 1;
  float best_ms = 1e30f;
  int r = SG_OK;
  for (int cand = 0; cand < 2 * nc && r == SG_OK; ++cand) {
    const int c = cands[cand % nc], pairs = cand < nc ? 1 : 0;
    const int maxo = (h->P + c - 1) / c;
    if (maxo > 8 || (c > 256 && maxo > 4)) continue;
    if (pairs && h->q >= 0) continue;
    t_out = c;
    p_out = pairs;
    r = launch_outer_matvec(h, a, s, df);
    if (r != SG_OK) break;
    cudaEventRecord(e0, s);
    for (int rep = 0; rep < 5 && r == SG_OK; ++rep) r = launch_outer_matvec(h, a, s, df);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r == SG_OK && ms < best_ms) {
      best_ms = ms;
      best = c;
      best_pairs = pairs;
    }
  }
  t_out = best;
  p_out = h->q >= 0 ? 0 : best_pairs;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return r;
}

// Tuned shapes per problem class: problems with the same device, sizes, chaos
// space and row lengths run the same launches, so a class is timed once per
// process and later handles of that class take its shapes without timing.
struct TuneKey {
  int dev, n, nnz, M, p, family, max_row, q, staged;
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, n, nnz, M, p, family, max_row, q, staged) <
           std::tie(o.dev, o.n, o.nnz, o.M, o.p, o.family, o.max_row, o.q, o.staged);
  }
};
struct TuneVal {
  int t64, t32, tout, p64, p32, pout, tdf, pdf;
  std::map<int, int> inner;   // FP32 batch width -> inner solver
};
static std::mutex g_tune_mu;
static std::map<TuneKey, TuneVal> g_tune_cache;

static TuneKey tune_key(const sg_problem* h) {
  return TuneKey{h->device, h->n, h->nnz, h->M, h->p, h->family, h->max_row_nnz, h->q, h->staged_pairs};
}

// A block size the product kernels are instantiated for: whole warps, 32 to
// 1024 threads, at most 8 outputs per thread (4 above 256 threads).
static bool valid_block(int threads, int P) {
  if (threads < 32 || threads > 1024 || threads % 32) return false;
  const int maxo = (P + threads - 1) / threads;
  return maxo <= (threads > 256 ? 4 : 8);
}

}  // namespace sghsc

using namespace sghsc;

extern "C" {

// The inner solver of each degree-level width, where several can run the
// batch (cluster solvers on grids up to 127^2): each candidate solves an FP32
// batch of that width (a constant right-hand side, two fixed PCG iterations,
// the default V-cycle) captured as a graph, timed over three replays after a
// first one; the fastest is kept for the width.
static int autotune_inner(sg_problem* h, cudaStream_t s) {
  if (!h->cl_plan) return SG_OK;
  std::vector<int> widths;
  for (int l = 0; l <= h->p; ++l) {
    const int w = h->off[l + 1] - h->off[l];
    if (w > 0 && std::find(widths.begin(), widths.end(), w) == widths.end()) widths.push_back(w);
  }
  const int wmax = *std::max_element(widths.begin(), widths.end());
  SG_TRY(ensure_inner_work(h, SG_F32, std::max(wmax, h->wmax)));   // no allocation under capture
  const size_t bytes = (size_t)h->n * wmax * sizeof(float);
  float *B = nullptr, *X = nullptr;
  SG_TRY_CUDA(cudaMalloc((void**)&B, bytes));
  cudaError_t ce = cudaMalloc((void**)&X, bytes);
  if (ce != cudaSuccess) {
    cudaFree(B);
    SG_TRY_CUDA(ce);
  }
  cudaMemsetAsync(B, 0x3f, bytes, s);   // every value 0.747f
  sg_prec_opts o;
  sg_default_prec_opts(&o);
  o.precision = SG_F32;
  o.inner_fixed_iters = 2;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int r = SG_OK;
  for (const int w : widths) {
    const std::vector<int> cands = inner_path_candidates(h, w);
    if (cands.size() < 2) continue;
    int best = cands[0];
    float best_ms = 1e30f;
    for (const int c : cands) {
      h->inner_pick[w] = c;
      clear_graphs(h);
      auto enq = [&](cudaStream_t cs) { return inner_solve(h, SG_F32, B, w, SG_F32, X, w, SG_F32, w, o, cs); };
      r = run_graph(h, "tune_inner", enq, s);
      if (r != SG_OK) break;
      cudaEventRecord(e0, s);
      for (int rep = 0; rep < 3 && r == SG_OK; ++rep) r = run_graph(h, "tune_inner", enq, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r == SG_OK && ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
    if (r != SG_OK) {
      h->inner_pick.erase(w);   // no choice left behind from a failed trial
      break;
    }
    h->inner_pick[w] = best;
  }
  clear_graphs(h);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(B);
  cudaFree(X);
  if (r == SG_OK) SG_TRY_CUDA(cudaGetLastError());
  return r;
}

int sg_autotune(sg_problem* h, void* stream) {
  set_error("");
  if (!h) {
    set_error("sg_autotune: null handle");
    return SG_ERR_INVALID_ARG;
  }
  clear_graphs(h);  // captured graphs hold the old launch shapes
  const TuneKey key = tune_key(h);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      const TuneVal& v = it->second;
      h->k1_threads[SG_F64] = v.t64;
      h->k1_threads[SG_F32] = v.t32;
      h->outer_threads = v.tout;
      h->k1_pairs[SG_F64] = v.p64;
      h->k1_pairs[SG_F32] = v.p32;
      h->outer_pairs = v.pout;
      h->outer_threads_df = v.tdf;
      h->outer_pairs_df = v.pdf;
      h->inner_pick = v.inner;
      return SG_OK;
    }
  }
  SG_TRY(autotune_k1(h, SG_F64, (cudaStream_t)stream));
  // the FP32 full product takes the row kernel (fixed shape) where it applies
  if (!rows32_usable(h, h->all, h->P, true)) SG_TRY(autotune_k1(h, SG_F32, (cudaStream_t)stream));
  SG_TRY(autotune_outer(h, (cudaStream_t)stream, false));
  // the double-float pair-form kernel has a fixed shape; tune the general one only when it stands in
  if (!df_pairs_usable(h, h->all, h->P)) SG_TRY(autotune_outer(h, (cudaStream_t)stream, true));
  SG_TRY(autotune_inner(h, (cudaStream_t)stream));
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[key] = TuneVal{h->k1_threads[SG_F64], h->k1_threads[SG_F32], h->outer_threads,
                              h->k1_pairs[SG_F64],   h->k1_pairs[SG_F32],   h->outer_pairs,
                              h->outer_threads_df,   h->outer_pairs_df,     h->inner_pick};
  return SG_OK;
}

int sg_autotune_set(sg_problem* h, int threads_f64, int threads_f32, int threads_outer, int pairs_f64,
                    int pairs_f32, int pairs_outer) {
  set_error("");
  if (!h) {
    set_error("sg_autotune_set: null handle");
    return SG_ERR_INVALID_ARG;
  }
  for (int t : {threads_f64, threads_f32, threads_outer})
    if (t != 0 && !valid_block(t, h->P)) {
      set_error("sg_autotune_set: block size %d not usable for P = %d", t, h->P);
      return SG_ERR_INVALID_ARG;
    }
  clear_graphs(h);
  h->k1_threads[SG_F64] = threads_f64;
  h->k1_threads[SG_F32] = threads_f32;
  h->outer_threads = threads_outer;
  h->k1_pairs[SG_F64] = pairs_f64 && h->q < 0 ? 1 : 0;   // gPC: gather form only
  h->k1_pairs[SG_F32] = pairs_f32 && h->q < 0 ? 1 : 0;
  h->outer_pairs = pairs_outer && h->q < 0 ? 1 : 0;
  h->outer_threads_df = threads_outer;      // the double-float variant takes the same shape
  h->outer_pairs_df = h->outer_pairs;
  return SG_OK;
}

int sg_autotune_outer_result(const sg_problem* h, int* threads_outer) {
  if (!h) {
    set_error("sg_autotune_outer_result: null handle");
    return SG_ERR_INVALID_ARG;
  }
  if (threads_outer) *threads_outer = h->outer_threads;
  return SG_OK;
}

int sg_autotune_forms(const sg_problem* h, int* pairs_f64, int* pairs_f32, int* pairs_outer) {
  if (!h) {
    set_error("sg_autotune_forms: null handle");
    return SG_ERR_INVALID_ARG;
  }
  if (pairs_f64) *pairs_f64 = h->k1_pairs[SG_F64];
  if (pairs_f32) *pairs_f32 = h->k1_pairs[SG_F32];
  if (pairs_outer) *pairs_outer = h->outer_pairs;
  return SG_OK;
}

int sg_autotune_result(const sg_problem* h, int* threads_f64, int* threads_f32) {
  if (!h) {
    set_error("sg_autotune_result: null handle");
    return SG_ERR_INVALID_ARG;
  }
  if (threads_f64) *threads_f64 = h->k1_threads[SG_F64];
  if (threads_f32) *threads_f32 = h->k1_threads[SG_F32];
  return SG_OK;
}

int sg_batch_create(int count, sg_problem* const* problems, sg_batch** out) {
  set_error("");
  if (!out) {
    set_error("sg_batch_create: out is null");
    return SG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (count < 1 || !problems) {
    set_error("sg_batch_create: invalid arguments");
    return SG_ERR_INVALID_ARG;
  }
  for (int i = 0; i < count; ++i) {
    bool bad = !problems[i];
    for (int j = 0; j < i && !bad; ++j) bad = problems[i] == problems[j];
    if (bad) {
      set_error("sg_batch_create: null or repeated handle at %d", i);
      return SG_ERR_INVALID_ARG;
    }
  }
  sg_batch* b = new sg_batch();
  b->hs.assign(problems, problems + count);
  b->branch.assign(count, nullptr);
  b->join.assign(count, nullptr);
  cudaError_t e = cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    set_error("sg_batch_create: %s", cudaGetErrorString(e));
    sg_batch_destroy(b);
    return SG_ERR_CUDA;
  }
  *out = b;
  return SG_OK;
}

static int check_batch_call(sg_batch* b, const double* const* F, double* const* U, const sg_solve_opts* opts) {
  if (!b || !F || !U || !opts) {
    set_error("sg_batch_solve: invalid arguments");
    return SG_ERR_INVALID_ARG;
  }
  if (opts->schur_reduced) {
    set_error("sg_batch_solve: the Schur-reduced system is solved by sg_solve only");
    return SG_ERR_UNSUPPORTED;
  }
  for (size_t i = 0; i < b->hs.size(); ++i)
    if (!F[i] || !U[i] || F[i] == U[i]) {
      set_error("sg_batch_solve: invalid buffers for system %zu", i);
      return SG_ERR_INVALID_ARG;
    }
  return SG_OK;
}

int sg_batch_solve(sg_batch* b, const double* const* F, double* const* U, const sg_solve_opts* opts,
                   sg_solve_stats* stats, void* stream) {
  set_error("");
  SG_TRY(check_batch_call(b, F, U, opts));
  return batch_solve(b, F, U, *opts, stats, (cudaStream_t)stream);
}

int sg_batch_solve_host(sg_batch* b, const double* const* F_host, double* const* U_host, const sg_solve_opts* opts,
                        sg_solve_stats* stats, void* stream) {
  set_error("");
  SG_TRY(check_batch_call(b, F_host, U_host, opts));
  return batch_solve(b, F_host, U_host, *opts, stats, (cudaStream_t)stream, true);
}

void sg_batch_destroy(sg_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  batch_clear(b);
  for (auto s : b->branch)
    if (s) cudaStreamDestroy(s);
  for (auto ev : b->join)
    if (ev) cudaEventDestroy(ev);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cs) cudaStreamDestroy(b->cs);
  delete b;
}

}  // extern "C"
