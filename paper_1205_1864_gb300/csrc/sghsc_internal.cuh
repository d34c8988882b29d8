// Internal declarations of libsghsc: the problem handle, device tables and
// the kernels' host-side launchers. Not part of the public C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "sghsc.h"

namespace sghsc {

void set_error(const char* fmt, ...);
// Process-wide count of kernel launches made by this library (sg_kernel_launches()).
void note_launch();
struct GraphEntry;
void clear_graphs(sg_problem* h);

#define SG_TRY_CUDA(call)                                                           \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      ::sghsc::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,                  \
                         cudaGetErrorString(e_));                                   \
      return e_ == cudaErrorMemoryAllocation ? SG_ERR_OOM : SG_ERR_CUDA;            \
    }                                                                               \
  } while (0)

#define SG_TRY(call)                    \
  do {                                  \
    int s_ = (call);                    \
    if (s_ != SG_OK) return s_;         \
  } while (0)

#define SG_CHECK_LAUNCH() SG_TRY_CUDA(cudaGetLastError())

// Bits of the device status word written by kernels.
enum : int {
  ST_INNER_NOT_SPD = 1,
  ST_INNER_MAXIT = 2,
  ST_OUTER_BREAKDOWN = 4,
};

// Sparse G coupling in gather form: for output chaos column l (local index in
// the output range), edges ptr[l]..ptr[l+1] with KL index k (1..M), input
// column j (local index in the input range) and coefficient c = (G_k)_{lj}.
struct EdgeList {
  int nout = 0, nedges = 0;
  int out0 = 0, in0 = 0, nin = 0;   // chaos columns [out0, out0 + nout) from [in0, in0 + nin)
  int* ptr = nullptr;
  int* perm = nullptr;   // thread slot -> output column, by coupling count (descending, stable)
  int* k = nullptr;
  int* j = nullptr;
  double* c64 = nullptr;
  float* c32 = nullptr;
  void* cdf = nullptr;   // the coefficients as double-float pairs (df64)
  // The distinct (k, j) of the couplings, ordered by k then j (a sum
  // sum_c a_k(r,c) U(c,j) serves every coupling with that pair), and the
  // pair of each coupling.
  int npair = 0;
  int* pk = nullptr;
  int* pj = nullptr;
  int* pair = nullptr;
  // Compact coupling table: pair << 8 | class per coupling, the coefficient of
  // class c in ctab[c] (df64). The coefficients of the linear KL expansion take
  // one value per 1-D degree, so a few classes cover them; ncls = 0 when the
  // table does not compress (more than 256 distinct coefficients).
  // couplings packed (pair << 8 | coefficient class), slot-transposed: the
  // c-th coupling of output slot s (perm order) at ctr[tb(s) + 32 c], so the
  // lanes of a warp (32 consecutive slots) read consecutive words; tb(s) is
  // in the slot's descriptor (sdesc)
  unsigned* ctr = nullptr;
  // the same positions packed as class << 24 | (k rows32_stride(nin) + j)
  // (below 2^24)
  unsigned* ckj = nullptr;
  int2* sdesc = nullptr;     // per slot: tb(s), output << 16 | couplings
  void* ctab = nullptr;      // df64
  float* ctab32 = nullptr;   // the same coefficients in FP32
  int ncls = 0;
};

// One grid of the geometric multigrid hierarchy: interior nodes nx*ny, x
// fastest; 9-point stencil [n][9], slot (dy+1)*3 + (dx+1), zero where the
// neighbour is outside the interior.
struct GridLevel {
  int nx = 0, ny = 0, n = 0;
  double* st_base = nullptr;   // stencil of A_0 as given to sg_setup (scale 1)
  double* st64 = nullptr;
  float* st32 = nullptr;
  double* dinv64 = nullptr;
  float* dinv32 = nullptr;
};

// Device control block of one batched inner solve.
struct InnerCtl {
  int it;            // batch iteration counter (selects the p ping-pong buffer)
  unsigned ticket;   // last-block detection of the reduction kernels
  int active;        // columns still iterating
  int pad;
};

// Workspace of the batched inner PCG / V-cycle for one element size; blocks
// are n_g x wcap packed, wcap the widest batch of one launch.
struct InnerWork {
  int wcap = 0;
  size_t esize = 0;
  void *x = nullptr, *r = nullptr, *z = nullptr, *zt = nullptr, *pA = nullptr, *pB = nullptr, *q = nullptr;
  std::vector<void*> cb, cx, cxt;         // per coarse grid g >= 1: rhs, iterate, ping-pong
  double* part = nullptr;                 // block partial sums [nblk][wcap]
  int part_blocks = 0;
  double *rho = nullptr, *pq = nullptr, *rr = nullptr, *bb = nullptr, *alpha = nullptr, *beta = nullptr;
  float *alphaf = nullptr, *betaf = nullptr;
  int *done = nullptr, *iters = nullptr;
  InnerCtl* ctl = nullptr;
};

// Device control block of the outer solve.
struct OuterCtl {
  int it;            // outer iterations done
  unsigned ticket;
  int maxit;
  int pad;
  double tol;
};

struct GraphEntry {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};

}  // namespace sghsc

struct sg_problem {
  int n = 0, nnz = 0, M = 0, p = 0, P = 0, family = 0;
  int q = -1;                         // -1: linear KL expansion; >= 0: gPC coefficient of total degree q
  int nterm = 0;                      // value terms per nonzero: M + 1, or C(M + q, M) for the gPC case
  int nx = 0, ny = 0;                 // mesh interior size (0 if no mesh)
  int device = 0, num_sms = 0;
  int smem_optin = 0;                 // shared memory a block may opt in to (bytes)
  std::vector<int> alpha;             // host P*M
  std::vector<int> off;               // host p+2
  // shared CSR pattern and KL values [nnz][M+1]
  int* rowptr = nullptr;
  int* colidx = nullptr;
  double* vals64 = nullptr;
  float* vals32 = nullptr;
  double* vals_base = nullptr;        // [nnz][M+1] as given to sg_setup (scales 1)
  void* vals_df = nullptr;            // [nnz][M+1] double-float pairs (df64) of vals64
  double* scales_dev = nullptr;       // current scale of each A_k
  std::vector<double> scales;         // host copy
  double* mass64 = nullptr;
  int max_row_nnz = 0;
  // G couplings: all edges (for the full operator) and per adjacent level pair
  sghsc::EdgeList all;                      // outputs 0..P-1, inputs 0..P-1
  std::vector<sghsc::EdgeList> pre;         // pre[l]:  out level l-1, in level l   (B_l), l = 1..p
  std::vector<sghsc::EdgeList> post;        // post[l]: out level l,   in level l-1 (C_l), l = 1..p
  sghsc::EdgeList sub;                      // levels 0..p-1 among themselves (A_{p-1}, Schur-reduced system)
  // gPC coefficient (q >= 0): B_l reaches every lower level and D_l is not block
  // diagonal; dlev[l] holds the couplings of level l with itself (i >= 1)
  std::vector<sghsc::EdgeList> dlev;
  std::vector<int> gamma;                   // host nterm*M: multi-indices of the coefficient terms
  // nested Krylov solves with D_l (gPC case): FP64 blocks n x wmax and their CG control
  double *lx = nullptr, *lr = nullptr, *lz = nullptr, *lp = nullptr, *lq = nullptr, *lb = nullptr;
  sghsc::OuterCtl* lctl = nullptr;
  double* lsc = nullptr;
  double *lhist_alpha = nullptr, *lhist_beta = nullptr, *lhist_res = nullptr;
  int lhist_cap = 0;
  double* fG = nullptr;                     // n x off[p] right-hand side g_{p-1} of the reduced system
  // multigrid
  std::vector<sghsc::GridLevel> grids;
  bool mg_full = false;                     // the hierarchy reaches the one-node grid (V-cycle usable)
  int cb_level = 0;                         // first grid handled by the in-block coarse V-cycle
  void* cl_plan = nullptr;                  // cluster inner solvers: plans and scratch (null: not usable)
  std::map<int, int> inner_pick;            // FP32 batch width -> inner solver chosen by the autotuner
  bool pipe_off = false;                    // SGHSC_NO_PIPE=1: no row-pipelined sweeps on large grids
  // workspace
  sghsc::InnerWork iw32, iw64;
  float* R32 = nullptr;                     // n x P working residual (mixed HSC)
  float* Z32 = nullptr;                     // n x P preconditioner output (mixed HSC)
  float* T32 = nullptr;                     // n x wmax packed post-correction rhs
  double* R64w = nullptr;                   // n x P working residual (FP64 HSC)
  double* T64 = nullptr;                    // n x wmax packed
  int wmax = 0;                             // widest degree level
  // outer solver (n x P FP64 each)
  double *fF = nullptr, *fx = nullptr, *fr = nullptr, *fz = nullptr, *fpA = nullptr, *fpB = nullptr, *fq = nullptr;
  double* opart = nullptr;                  // [nblk][2] partial dots
  int opart_blocks = 0;
  double* osc = nullptr;                    // device scalars
  double* osc_host = nullptr;               // pinned mirror
  sghsc::OuterCtl* octl = nullptr;
  double *hist_alpha = nullptr, *hist_beta = nullptr, *hist_res = nullptr;
  // staging for the standalone inner-solve entry point
  void *io_in = nullptr, *io_out = nullptr;
  size_t io_bytes = 0;
  int* status = nullptr;                    // device status word
  int* status_host = nullptr;               // pinned
  long long* iacc = nullptr;                // device: [total inner iterations, max per column]
  double* wdev = nullptr;                   // device copy of gradient weights
  int wdev_cap = 0;
  // graphs
  cudaStream_t cap[4] = {nullptr, nullptr, nullptr, nullptr};
  int cap_depth = 0;
  bool capturing = false;
  bool eager = false;                       // SGHSC_EAGER=1: host-driven loops, no graphs
  int loop_depth = 0;
  int* loopflags = nullptr;                 // device: loop condition per nesting depth (eager mode)
  int* loopflag_host = nullptr;             // pinned
  std::map<std::string, sghsc::GraphEntry> graphs;
  // autotuned block sizes of the full SG product (0: heuristic), per element type
  int k1_threads[2] = {0, 0};
  int outer_threads = 0;                    // block size of the fused outer product (0: 256)
  int k1_pairs[2] = {1, 1};                 // full SG product in pair form (1) or gather form (0)
  int outer_pairs = 1;                      // the same for the fused outer product
  int outer_threads_df = 0;                 // block size and form of its double-float variant
  int outer_pairs_df = 1;
  int staged_pairs = 1;                     // the staged pair kernels of dfprod.cu where usable
  long long ws_gen = 0;                     // bumped whenever captured graphs become invalid
};

namespace sghsc {

// Accumulation type code of launch_block_matvec beside SG_F64 / SG_F32:
// double-float pairs on the FP32 units (df64.cuh).
enum { ACC_DF64 = 16 };

// ---- launchers (matvec.cu) ----
// Generic block product used for the full operator (K1) and the level products (K2):
//   Y[r, l] = beta * Yin[r, l] + alpha * ( diag ? sum_c a_0(r,c) X[c, l] : 0
//                                          + sum_{(k,j,c)} c sum_c' a_k(r,c') X[c', j] )
// TIn: element type of X; TAcc: arithmetic and value type; TB: type of Yin; TO: type of Y.
int launch_block_matvec(sg_problem* h, int tin, int tacc, int tb, int tout, const void* X, int ldx,
                        int wx, const EdgeList& E, bool diag, const void* Yin, int ldyin,
                        double alpha, double beta, void* Y, int ldy, cudaStream_t s);

// ---- double-float pair-form products (dfprod.cu) ----
// The input block holds FP32 values; usable when the pairs and the staging fit.
bool df_pairs_usable(const sg_problem* h, const EdgeList& E, int wx);
// Y = sum_k A_k U G_k^T: U FP32, double-float sums, Y FP64.
int launch_df_apply(sg_problem* h, const float* U, double* Y, cudaStream_t s);
// Y = Yin - sum_k A_k X G_k[out, in]^T: X FP32, Yin FP64, Y FP32.
int launch_df_level(sg_problem* h, const EdgeList& E, const float* X, int ldx, int wx, const double* Yin, int ldyin,
                    float* Y, int ldy, cudaStream_t s);
// Level products with at most 16 output columns and fewer than 512 input
// columns, one thread per (row, output) (levelnarrow.cu): Y = Yin - sum
// (Yin may alias Y).
bool narrow_usable(const sg_problem* h, const EdgeList& E, int wx);
template <typename T>
int launch_level_narrow(sg_problem* h, const EdgeList& E, const T* X, int ldx, const T* Yin, int ldyin, T* Y, int ldy,
                        cudaStream_t s);
// Row stride of the term sums of the FP32 row kernel (rows32.cu).
constexpr int ROWS32_COLS = 512;   // input columns per pass of a block (two per thread)
__host__ __device__ constexpr int rows32_stride(int wx) { return (wx + ROWS32_COLS - 1) / ROWS32_COLS * ROWS32_COLS; }
// FP32 products with the input columns in registers (rows32.cu): usable and
// preferred for E (compact table, sizes, inputs at least 512 columns wide).
bool rows32_usable(const sg_problem* h, const EdgeList& E, int wx, bool diag);
int launch_rows32(sg_problem* h, const EdgeList& E, bool diag, const float* X, int ldx, int wx, const float* Yin,
                  int ldyin, float* Y, int ldy, cudaStream_t s);

// ---- inner solver (inner.cu) ----
int ensure_inner_work(sg_problem* h, int dtype, int wcap);
void free_inner_work(sg_problem* h);
int inner_vcycle(sg_problem* h, int dtype, const void* B, void* X, int w, const sg_prec_opts& o,
                 cudaStream_t s);
// Solve A_0 X = B columnwise inside a graph capture on s. B read from src
// (ld_src, element type src_t), solution written to dst (ld_dst, type dst_t).
int inner_solve(sg_problem* h, int dtype, const void* src, int ld_src, int src_t, void* dst,
                int ld_dst, int dst_t, int w, const sg_prec_opts& o, cudaStream_t s);
int check_prec_opts(const sg_prec_opts& o);
// M_0 alone (one V-cycle, or the diagonal) on w strided columns, same type in and out.
int m0_apply(sg_problem* h, int dtype, const void* src, int lds, void* dst, int ldd, int w, const sg_prec_opts& o,
             cudaStream_t s);
// The inner solves of o can run on h (grids for the diagonal M_0, the whole
// hierarchy for the V-cycle); sets the error message and returns
// SG_ERR_UNSUPPORTED otherwise.
int check_inner_support(const sg_problem* h, const sg_prec_opts& o, const char* name);

// ---- cluster-resident inner solver (inner_cluster.cu) ----
// Plan the on-chip hierarchy after the grids are built (leaves cl_plan null
// when the hierarchy does not fit, or SGHSC_NO_CLUSTER=1).
int cluster_setup(sg_problem* h);
void cluster_free(sg_problem* h);
// True when an FP32 batch of w columns takes the cluster solver.
bool cluster_usable(const sg_problem* h, int dtype, int w);
// The inner solvers an FP32 batch of w columns may take (0 the stand-alone
// kernels, 1 / 3 the on-chip cluster solver with 8 / 16 CTAs, 2 the wide one).
std::vector<int> inner_path_candidates(const sg_problem* h, int w);
// inner_solve for FP32 on a usable handle: one cluster launch per solve.
int inner_solve_cluster(sg_problem* h, const void* src, int ld_src, int src_t, void* dst, int ld_dst, int dst_t,
                        int w, const sg_prec_opts& o, cudaStream_t s);

// ---- HSC / mean preconditioner (hsc.cu) ----
int prepare_precond(sg_problem* h, int kind, const sg_prec_opts& o);
// With o.precision == SG_F32 a null Z leaves the result in h->Z32 (FP32)
// without widening it (the outer solver then reads z there).
int hsc_apply_impl(sg_problem* h, const double* R, double* Z, const sg_prec_opts& o, cudaStream_t s);
int mean_apply_impl(sg_problem* h, const double* R, double* Z, const sg_prec_opts& o, cudaStream_t s);
int bgs_apply_impl(sg_problem* h, const double* R, double* Z, const sg_prec_opts& o, cudaStream_t s);
// The same on the hierarchy of levels 0..p with leading dimension P (the
// Schur-reduced system uses p = h->p - 1 and P = h->off[h->p]).
int hsc_apply_lv(sg_problem* h, const double* R, double* Z, const sg_prec_opts& o, cudaStream_t s, int p, int P);
int bgs_apply_lv(sg_problem* h, const double* R, double* Z, const sg_prec_opts& o, cudaStream_t s, int p, int P);
int mean_apply_lv(sg_problem* h, const double* R, double* Z, const sg_prec_opts& o, cudaStream_t s, int P);

// ---- outer solver (fcg.cu) ----
int ensure_outer(sg_problem* h);
int solve_prepare(sg_problem* h, const sg_solve_opts& o);
std::string solve_key(const sg_solve_opts& o);
int solve_stage_in(sg_problem* h, const double* F, const double* U, const sg_solve_opts& o, cudaStream_t s);
// the whole solve (device-controlled loops), enqueued on a capturing stream
int enqueue_solve(sg_problem* h, const sg_solve_opts& o, cudaStream_t s);
int solve_collect(sg_problem* h, const sg_solve_opts& o, sg_solve_stats* st, double wall_ms);
int check_solve_opts(const sg_problem* h, const sg_solve_opts* opts);

// ---- small elementwise kernels (vec.cu) ----
// n doubles between a host block (src when to_device, else dst) and a device
// block: page-locked host memory by a kernel through its device mapping,
// other host memory by cudaMemcpyAsync (fcg.cu)
int copy_host(sg_problem* h, const double* src, double* dst, size_t n, bool to_device, cudaStream_t s);
// dst = src, n doubles, by a kernel (either side may be page-locked host memory)
int launch_copy64(const double* src, double* dst, long long n, int num_sms, cudaStream_t s);
int launch_cast(const void* src, int src_t, int lds, void* dst, int dst_t, int ldd, int rows,
                int cols, cudaStream_t s);

std::string opts_key(const sg_prec_opts& o);

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace sghsc
