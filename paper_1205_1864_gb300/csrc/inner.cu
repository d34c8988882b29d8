// K3 + K4: the batched inner PCG on the mean-value matrix A_0 with a
// geometric multigrid V-cycle as its preconditioner M_0.
//
// Sec. 5: the diagonal blocks D_l are block diagonal with copies of A_0 (the
// Lemma of Sec. 3), so their inverses are many independent solves with A_0;
// Sec. 5 replaces exact solves by "independent loops of preconditioned Krylov
// subspace iterations". Here all columns of one level form one batch: each
// kernel walks an n x w node-major block (column index fastest, so a warp
// reads consecutive columns of one node and the stencil coefficients of that
// node are loaded once for all its columns). Each column keeps its own CG
// scalars and a done flag; a column is finished when ||r|| <= tol ||b||
// (zero columns at entry), and finished columns are skipped by every kernel.
//
// Thread mapping: a block has k*w threads (k = max(1, 1024 / w)), thread t
// always handles column t mod w and nodes (blockIdx*k + t / w) + m * grid*k,
// so per-column partial sums are register accumulations followed by a
// fixed-order block reduction; the last block to finish a reduction kernel
// sums the block partials in block order and updates the CG scalars, so the
// results do not depend on scheduling and no separate finalisation launch is
// needed. The iteration loop is a CUDA graph WHILE node whose condition the
// convergence kernel sets (graph.cu).
//
// V-cycle kernels (weighted Jacobi, nu sweeps before and after, bilinear
// transfers, Galerkin coarse operators built in setup.cu):
//   k_smooth00        two sweeps from a zero iterate in one pass
//   k_resid_restrict  the residual b - A x formed on the fly and restricted
//   k_prolong_jacobi  the coarse correction interpolated on the fly and the
//                     first post-smoothing sweep applied to it
//   k_jacobi          further sweeps; the last sweep of the finest grid also
//                     reduces r . z for the CG
//   k_vcycle_coarse   all grids with <= 1024 nodes: one 1024-thread block per column
//                     runs the rest of the V-cycle in shared memory.
#include <algorithm>
#include <mutex>

#include "graph.cuh"
#include "sghsc_internal.cuh"

namespace sghsc {

constexpr int MAX_LEVELS = 16;

struct Shape {
  int w, k, bdim, grid;
};

// k*w threads per block (up to 1024), at most `per_sm` blocks per SM. The
// reduction kernels use one block per SM: few block partials per column, so
// the last-block reduction stays short.
static Shape make_shape(const sg_problem* h, int nodes, int w, int per_sm = 2) {
  Shape s;
  s.w = w;
  s.k = std::max(1, 1024 / w);
  s.bdim = s.k * w;
  s.grid = std::max(1, std::min(ceil_div(nodes, s.k), h->num_sms * per_sm));
  return s;
}

template <typename T>
struct Acc;
template <>
struct Acc<float> {
  using type = float;
};
template <>
struct Acc<double> {
  using type = double;
};

enum { FIN_INIT = 0, FIN_RHO = 1, FIN_ALPHA = 2, FIN_CONV = 3 };

struct FinArgs {
  void* part;        // block partials [nblk][ldp] in the solver's accumulation type
  int ldp;
  InnerCtl* ctl;
  double *rho, *pq, *rr, *bb, *alpha, *beta;
  float *alphaf, *betaf;  // FP32 copies read by the FP32 kernels
  int *done, *iters;
  int* status;
  double tol2;
  int maxit, fixed;
  cudaGraphConditionalHandle cond;
  int has_cond;
  int* flag;
  long long* iacc;  // running [total, max] of per-column iteration counts
};

__device__ __forceinline__ void thread_pos(int w, int k, int& col, int& node0, int& nstep) {
  col = threadIdx.x % w;
  node0 = blockIdx.x * k + threadIdx.x / w;
  nstep = gridDim.x * k;
}

// Lanes per column group: the largest power of two g <= 32 with g*w <= bdim.
// Column c is reduced by the g consecutive threads c*g .. c*g+g-1, which lie in
// one warp, so a group finishes with g-wide shuffles (fixed order, no block
// barrier); threads beyond w*g only take part in the shuffles.
__device__ __forceinline__ int group_lanes(int w, int bdim) {
  int g = 1;
  while (g < 32 && 2 * g * w <= bdim) g *= 2;
  return g;
}

template <typename A>
__device__ __forceinline__ A group_shfl_sum(A s, int g) {
  for (int o = g >> 1; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, g);
  return s;
}

// True for a warp that owns at least one column of the lane-group layout
// (warp-uniform); the other warps skip the column arithmetic, which matters
// because FP64 instructions issue at a fraction of the FP32 rate.
__device__ __forceinline__ bool warp_owns_column(int w, int g) { return (int)((threadIdx.x & ~31u) / g) < w; }

// Per-column block partial of the k threads of each column (thread t holds
// column t mod w, slice t / w), summed in the accumulation type A of the
// solver (FP32 for the FP32 inner solves) and stored as a double.
template <typename A>
__device__ __forceinline__ void block_col_reduce(A v, int w, int k, A* part, int ldp) {
  __shared__ A red[1024];
  red[threadIdx.x] = v;
  __syncthreads();
  const int g = group_lanes(w, blockDim.x);
  if (!warp_owns_column(w, g)) return;
  const int c = threadIdx.x / g, lane = threadIdx.x - c * g;
  A s = A(0);
  if (c < w)
    for (int j = lane; j < k; j += g) s += red[j * w + c];
  s = group_shfl_sum(s, g);
  if (c < w && lane == 0) {
    part[(size_t)blockIdx.x * ldp + c] = s;
    __threadfence();  // only the writers of partials need the release fence
  }
}

// True in the last block to finish (threadFenceReduction pattern): the writers
// of block partials have fenced; thread 0 takes a ticket, and the block whose
// ticket is the last one reads every partial from L2.
__device__ __forceinline__ bool last_block(unsigned* ticket) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    if (last) __threadfence();
  }
  __syncthreads();
  return last;
}

// Column-wise CG scalar updates from the block partials (last block only).
// Column c is summed by its lane group in the accumulation type A (blocks lane,
// lane + g, ... with four interleaved accumulators, then the g-wide shuffle);
// the column totals go through shared memory to threads 0..w-1, which update
// the scalars in FP64 (so only the first ceil(w/32) warps issue FP64 work).
// The order is fixed, so results are reproducible.
template <typename A>
__device__ void fin_columns(const FinArgs& f, int op, int w, int k, int nblk) {
  __shared__ int cnt;
  __shared__ double colsum[1024];
  if (threadIdx.x == 0) cnt = 0;
  const A* part = (const A*)f.part;
  const int g = group_lanes(w, blockDim.x);
  const int gc = threadIdx.x / g, lane = threadIdx.x - gc * g;
  if (warp_owns_column(w, g)) {
    A s0 = A(0), s1 = A(0), s2 = A(0), s3 = A(0);
    if (gc < w) {
      int b = lane;
      for (; b + 3 * g < nblk; b += 4 * g) {
        s0 += __ldcg(&part[(size_t)b * f.ldp + gc]);
        s1 += __ldcg(&part[(size_t)(b + g) * f.ldp + gc]);
        s2 += __ldcg(&part[(size_t)(b + 2 * g) * f.ldp + gc]);
        s3 += __ldcg(&part[(size_t)(b + 3 * g) * f.ldp + gc]);
      }
      for (; b < nblk; b += g) s0 += __ldcg(&part[(size_t)b * f.ldp + gc]);
    }
    const A s = group_shfl_sum((s0 + s1) + (s2 + s3), g);
    if (gc < w && lane == 0) colsum[gc] = (double)s;
  }
  __syncthreads();
  const int c = threadIdx.x;
  if (c < w) {
    const double s = colsum[c];
    if (op == FIN_INIT) {
      f.bb[c] = s;
      f.done[c] = !(s > 0.0);
      f.iters[c] = 0;
      f.beta[c] = 0.0;
      f.betaf[c] = 0.0f;
    } else if (!f.done[c]) {
      if (op == FIN_RHO) {
        f.beta[c] = f.iters[c] == 0 ? 0.0 : s / f.rho[c];
        f.betaf[c] = (float)f.beta[c];
        f.rho[c] = s;
      } else if (op == FIN_ALPHA) {
        f.pq[c] = s;
        if (!(s > 0.0)) {
          atomicOr(f.status, ST_INNER_NOT_SPD);
          f.alpha[c] = 0.0;
          f.done[c] = 1;
        } else {
          f.alpha[c] = f.rho[c] / s;
        }
        f.alphaf[c] = (float)f.alpha[c];
      } else if (op == FIN_CONV) {
        f.rr[c] = s;
        const int it = ++f.iters[c];
        bool fin;
        if (f.fixed > 0) {
          fin = it >= f.fixed;
        } else {
          fin = s <= f.tol2 * f.bb[c];
          if (!fin && it >= f.maxit) {
            fin = true;
            atomicOr(f.status, ST_INNER_MAXIT);
          }
        }
        if (!(s == s)) {  // non-finite residual: stop the column and flag it
          fin = true;
          atomicOr(f.status, ST_INNER_NOT_SPD);
        }
        f.done[c] = fin;
        if (fin) {
          atomicAdd((unsigned long long*)&f.iacc[0], (unsigned long long)it);
          atomicMax(&f.iacc[1], (long long)it);
        }
      }
    }
    if (!f.done[c]) atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (op == FIN_INIT) f.ctl->it = 0;
    if (op == FIN_CONV) f.ctl->it += 1;
    f.ctl->active = cnt;
    if (op == FIN_INIT || op == FIN_CONV) {
      if (f.has_cond) cudaGraphSetConditional(f.cond, cnt > 0 ? 1u : 0u);
      if (f.flag) *f.flag = cnt > 0;
    }
    f.ctl->ticket = 0;
  }
}

template <typename A>
__device__ __forceinline__ void reduce_finalize(const FinArgs& f, A v, int w, int k, int op) {
  block_col_reduce(v, w, k, (A*)f.part, f.ldp);
  if (last_block(&f.ctl->ticket)) fin_columns<A>(f, op, w, k, gridDim.x);
}

// (P xc) at fine node (fx, fy): bilinear interpolation from the coarse grid,
// coarse node (X, Y) sitting on fine node (2X+1, 2Y+1), zero outside.
template <typename T>
__device__ __forceinline__ T prolong_at(int fx, int fy, int nxc, int nyc, const T* __restrict__ xc, int w, int col) {
  int Xs[2], Ys[2];
  T wx[2], wy[2];
  int nxs, nys;
  if (fx & 1) { Xs[0] = (fx - 1) >> 1; wx[0] = T(1); nxs = 1; }
  else { Xs[0] = (fx >> 1) - 1; Xs[1] = fx >> 1; wx[0] = wx[1] = T(0.5); nxs = 2; }
  if (fy & 1) { Ys[0] = (fy - 1) >> 1; wy[0] = T(1); nys = 1; }
  else { Ys[0] = (fy >> 1) - 1; Ys[1] = fy >> 1; wy[0] = wy[1] = T(0.5); nys = 2; }
  T acc = T(0);
  for (int iy = 0; iy < nys; ++iy) {
    if (Ys[iy] < 0 || Ys[iy] >= nyc) continue;
    for (int ix = 0; ix < nxs; ++ix) {
      if (Xs[ix] < 0 || Xs[ix] >= nxc) continue;
      acc += wy[iy] * wx[ix] * xc[(size_t)(Ys[iy] * nxc + Xs[ix]) * w + col];
    }
  }
  return acc;
}

// A thread's node sequence node0, node0 + nstep, ... with the grid coordinates
// (x, y) kept incrementally (no division per node).
struct NodeIter {
  int node, x, y, nstep, dxs, dys, nx;
  __device__ __forceinline__ NodeIter(int node0, int step, int nx_) : node(node0), nstep(step), nx(nx_) {
    y = node0 / nx_;
    x = node0 - y * nx_;
    dys = step / nx_;
    dxs = step - dys * nx_;
  }
  __device__ __forceinline__ void next() {
    node += nstep;
    x += dxs;
    y += dys;
    if (x >= nx) {
      x -= nx;
      ++y;
    }
  }
};

// sum_j a_ij val(e_j, j, dy, dx) over the 9-point stencil of node (x, y),
// e_j = i + dy*rs + dx*w the element index of neighbour j = node + dy*nx + dx
// (node-major blocks, rs = nx*w). Interior nodes take a branch-free path.
template <typename T, typename F>
__device__ __forceinline__ T stencil9(const T* __restrict__ s9, int i, int rs, int w, int node, int x, int y, int nx,
                                      int ny, F val) {
  T acc = T(0);
  if (x > 0 && x < nx - 1 && y > 0 && y < ny - 1) {
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx)
        acc += s9[(dy + 1) * 3 + (dx + 1)] * val(i + dy * rs + dx * w, node + dy * nx + dx, dy, dx);
    return acc;
  }
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
    if (y + dy < 0 || y + dy >= ny) continue;
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      if (x + dx < 0 || x + dx >= nx) continue;
      acc += s9[(dy + 1) * 3 + (dx + 1)] * val(i + dy * rs + dx * w, node + dy * nx + dx, dy, dx);
    }
  }
  return acc;
}

// ---------------------------------------------------------------- V-cycle ---

// one sweep from zero: x = omega D^{-1} b
template <typename T>
__global__ void __launch_bounds__(1024) k_smooth0(int n, int w, int k, const T* __restrict__ dinv,
                                                  const T* __restrict__ b, T* __restrict__ x, T om,
                                                  const int* __restrict__ done) {
  int col, node, nstep;
  thread_pos(w, k, col, node, nstep);
  if (done[col]) return;
  for (; node < n; node += nstep) {
    const int i = node * w + col;
    x[i] = om * dinv[node] * b[i];
  }
}

// two sweeps from zero: x1 = omega D^{-1} b, x2 = x1 + omega D^{-1} (b - A x1)
template <typename T>
__global__ void __launch_bounds__(1024) k_smooth00(int nx, int ny, int w, int k, const T* __restrict__ st,
                                                   const T* __restrict__ dinv, const T* __restrict__ b,
                                                   T* __restrict__ x, T om, const int* __restrict__ done) {
  int col, node0, nstep;
  thread_pos(w, k, col, node0, nstep);
  if (done[col]) return;
  const int n = nx * ny, rs = nx * w;
  for (NodeIter it(node0, nstep, nx); it.node < n; it.next()) {
    const int i = it.node * w + col;
    const T ax1 = om * stencil9(st + it.node * 9, i, rs, w, it.node, it.x, it.y, nx, ny,
                                [&](int e, int j, int, int) { return dinv[j] * b[e]; });
    const T bi = b[i], di = dinv[it.node];
    x[i] = om * di * bi + om * di * (bi - ax1);
  }
}

// xo = xi + omega D^{-1} (b - A xi); with DOT also the partials of b . xo and FIN_RHO
template <typename T, bool DOT>
__global__ void __launch_bounds__(1024) k_jacobi(int nx, int ny, int w, int k, const T* __restrict__ st,
                                                 const T* __restrict__ dinv, const T* __restrict__ b,
                                                 const T* __restrict__ xi, T* __restrict__ xo, T om, FinArgs f) {
  int col, node0, nstep;
  thread_pos(w, k, col, node0, nstep);
  typename Acc<T>::type acc = 0;
  if (!f.done[col]) {
    const int n = nx * ny, rs = nx * w;
    for (NodeIter it(node0, nstep, nx); it.node < n; it.next()) {
      const int i = it.node * w + col;
      const T bi = b[i];
      const T ax = stencil9(st + it.node * 9, i, rs, w, it.node, it.x, it.y, nx, ny,
                            [&](int e, int, int, int) { return xi[e]; });
      const T v = xi[i] + om * dinv[it.node] * (bi - ax);
      xo[i] = v;
      if (DOT) acc += bi * v;
    }
  }
  if (DOT) reduce_finalize(f, acc, w, k, FIN_RHO);
}

// bc = P^T (b - A x): coarse node (X, Y) gathers the 3x3 fine residuals around (2X+1, 2Y+1)
template <typename T>
__global__ void __launch_bounds__(1024) k_resid_restrict(int nxf, int nyf, int nxc, int nyc, int w, int k,
                                                         const T* __restrict__ st, const T* __restrict__ b,
                                                         const T* __restrict__ x, T* __restrict__ bc,
                                                         const int* __restrict__ done) {
  int col, node0, nstep;
  thread_pos(w, k, col, node0, nstep);
  if (done[col]) return;
  const int n = nxc * nyc, rsf = nxf * w;
  for (NodeIter it(node0, nstep, nxc); it.node < n; it.next()) {
    const int cx = 2 * it.x + 1, cy = 2 * it.y + 1;
    T acc = T(0);
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const T wy = dy == 0 ? T(1) : T(0.5);
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const T wx = dx == 0 ? T(1) : T(0.5);
        const int fx = cx + dx, fy = cy + dy, fn = fy * nxf + fx;
        const int fi = fn * w + col;
        const T ax = stencil9(st + fn * 9, fi, rsf, w, fn, fx, fy, nxf, nyf,
                              [&](int e, int, int, int) { return x[e]; });
        acc += wx * wy * (b[fi] - ax);
      }
    }
    bc[it.node * w + col] = acc;
  }
}

// x' = x + P xc (on the fly), xo = x' + omega D^{-1} (b - A x'); DOT as k_jacobi.
// The coarse values that the 3x3 fine neighbourhood of (x0, y) interpolates
// from lie in the 3x3 coarse patch X in [Xb-1, Xb+1], Xb = floor((x0-1)/2)
// (same in y). Interpolation is separable with parity-dependent weights:
// even x0 -> offsets -1, 0, +1 read patch columns (1), (1,2)/2, (2);
// odd x0  -> (0,1)/2, (1), (1,2)/2.
template <typename T, bool DOT>
__global__ void __launch_bounds__(1024) k_prolong_jacobi(int nxf, int nyf, int nxc, int nyc, int w, int k,
                                                         const T* __restrict__ st, const T* __restrict__ dinv,
                                                         const T* __restrict__ b, const T* __restrict__ x,
                                                         const T* __restrict__ xc, T* __restrict__ xo, T om,
                                                         FinArgs f) {
  int col, node0, nstep;
  thread_pos(w, k, col, node0, nstep);
  typename Acc<T>::type acc = 0;
  if (!f.done[col]) {
    const int n = nxf * nyf, rs = nxf * w;
    const T h = T(0.5);
    for (NodeIter it(node0, nstep, nxf); it.node < n; it.next()) {
      const int Xb = (it.x - 1) >> 1, Yb = (it.y - 1) >> 1;
      T cp[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int Y = Yb - 1 + a;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int X = Xb - 1 + c;
          cp[a][c] = (Y >= 0 && Y < nyc && X >= 0 && X < nxc) ? xc[(Y * nxc + X) * w + col] : T(0);
        }
      }
      T tx[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (it.x & 1) {
          tx[a][0] = h * (cp[a][0] + cp[a][1]);
          tx[a][1] = cp[a][1];
          tx[a][2] = h * (cp[a][1] + cp[a][2]);
        } else {
          tx[a][0] = cp[a][1];
          tx[a][1] = h * (cp[a][1] + cp[a][2]);
          tx[a][2] = cp[a][2];
        }
      }
      T I[3][3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (it.y & 1) {
          I[0][d] = h * (tx[0][d] + tx[1][d]);
          I[1][d] = tx[1][d];
          I[2][d] = h * (tx[1][d] + tx[2][d]);
        } else {
          I[0][d] = tx[1][d];
          I[1][d] = h * (tx[1][d] + tx[2][d]);
          I[2][d] = tx[2][d];
        }
      }
      const int i = it.node * w + col;
      const T ax = stencil9(st + it.node * 9, i, rs, w, it.node, it.x, it.y, nxf, nyf,
                            [&](int e, int, int dy, int dx) { return x[e] + I[dy + 1][dx + 1]; });
      const T xi = x[i] + I[1][1];
      const T bi = b[i];
      const T v = xi + om * dinv[it.node] * (bi - ax);
      xo[i] = v;
      if (DOT) acc += bi * v;
    }
  }
  if (DOT) reduce_finalize(f, acc, w, k, FIN_RHO);
}

struct CoarseGrids {
  int g0, G;
  int nx[MAX_LEVELS], ny[MAX_LEVELS], off[MAX_LEVELS];
  const void* st[MAX_LEVELS];
  const void* dinv[MAX_LEVELS];
};

// The V-cycle from grid g0 down, one column per 1024-thread block (the coarse
// grids are latency-bound, so the work spreads over as many SMs as there are
// columns), entirely in shared memory: per grid a right-hand side, an iterate
// and a ping-pong buffer, plus every coarse stencil and inverse diagonal
// (staged once per block with independent loads in flight). Grids of at most
// 64 nodes are run by warp 0 alone with warp-level synchronisation.
template <typename T>
__device__ __forceinline__ void stage_copy(T* __restrict__ dst, const T* __restrict__ src, int count) {
  constexpr int U = 8;
  for (int base = 0; base < count; base += U * (int)blockDim.x) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * blockDim.x + threadIdx.x;
      v[u] = idx < count ? src[idx] : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * blockDim.x + threadIdx.x;
      if (idx < count) dst[idx] = v[u];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_vcycle_coarse(CoarseGrids L, int tot, int w, const T* __restrict__ bg,
                                                        T* __restrict__ xg, T om, int nu,
                                                        const int* __restrict__ done) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* sst = sm + 3 * tot;          // stencils [node][9] of all coarse grids
  T* sdi = sst + 9 * tot;         // inverse diagonals
  const int col = blockIdx.x;
  if (done[col]) return;
  const int tid = threadIdx.x;
  for (int g = L.g0; g < L.G; ++g) {
    const int n = L.nx[g] * L.ny[g];
    stage_copy(sst + 9 * L.off[g], (const T*)L.st[g], 9 * n);
    stage_copy(sdi + L.off[g], (const T*)L.dinv[g], n);
  }
  auto B = [&](int g) { return sm + 3 * L.off[g]; };
  auto Xa = [&](int g) { return sm + 3 * L.off[g] + L.nx[g] * L.ny[g]; };
  auto Xb = [&](int g) { return sm + 3 * L.off[g] + 2 * L.nx[g] * L.ny[g]; };
  auto sdot = [&](const T* s9, int nx, int ny, int x, int y, const T* v) {
    T acc = T(0);
    for (int dy = -1; dy <= 1; ++dy) {
      const int yy = y + dy;
      if (yy < 0 || yy >= ny) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int xx = x + dx;
        if (xx < 0 || xx >= nx) continue;
        acc += s9[(dy + 1) * 3 + (dx + 1)] * v[yy * nx + xx];
      }
    }
    return acc;
  };
  // grid g runs in warp mode (warp 0 only, __syncwarp) when it has <= 64 nodes
  auto wmode = [&](int g) { return L.nx[g] * L.ny[g] <= 64; };
  auto lsync = [&](bool wm) {
    if (wm) __syncwarp(); else __syncthreads();
  };
  {
    const int n0 = L.nx[L.g0] * L.ny[L.g0];
    T* b0 = B(L.g0);
    for (int idx = tid; idx < n0; idx += blockDim.x) b0[idx] = bg[idx * w + col];
  }
  __syncthreads();
  T* cur[MAX_LEVELS];
  T* oth[MAX_LEVELS];
  for (int g = L.g0; g < L.G; ++g) {
    const int nx = L.nx[g], ny = L.ny[g], n = nx * ny;
    const bool wm = wmode(g);
    const int lim = wm ? 32 : (int)blockDim.x;
    const bool act = tid < lim;
    const T* st = sst + 9 * L.off[g];
    const T* dinv = sdi + L.off[g];
    const T* b = B(g);
    T* c = Xa(g);
    T* o = Xb(g);
    if (g == L.G - 1) {  // coarsest grid (one node for square grids): exact solve
      if (act)
        for (int idx = tid; idx < n; idx += lim) c[idx] = dinv[idx] * b[idx];
      lsync(wm);
      cur[g] = c;
      oth[g] = o;
      break;
    }
    if (act)
      for (int idx = tid; idx < n; idx += lim) c[idx] = om * dinv[idx] * b[idx];
    lsync(wm);
    for (int s = 1; s < nu; ++s) {
      if (act)
        for (int idx = tid; idx < n; idx += lim) {
          const int y = idx / nx, x = idx - y * nx;
          o[idx] = c[idx] + om * dinv[idx] * (b[idx] - sdot(st + idx * 9, nx, ny, x, y, c));
        }
      lsync(wm);
      T* t = c; c = o; o = t;
    }
    if (act)
      for (int idx = tid; idx < n; idx += lim) {
        const int y = idx / nx, x = idx - y * nx;
        o[idx] = b[idx] - sdot(st + idx * 9, nx, ny, x, y, c);
      }
    lsync(wm);
    const int nxc = L.nx[g + 1], nyc = L.ny[g + 1];
    T* bc = B(g + 1);
    if (act)
      for (int idx = tid; idx < nxc * nyc; idx += lim) {
        const int Y = idx / nxc, X = idx - Y * nxc;
        T acc = T(0);
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const T wgt = (dx == 0 ? T(1) : T(0.5)) * (dy == 0 ? T(1) : T(0.5));
            acc += wgt * o[(2 * Y + 1 + dy) * nx + (2 * X + 1 + dx)];
          }
        bc[idx] = acc;
      }
    lsync(wm);
    cur[g] = c;
    oth[g] = o;
  }
  for (int g = L.G - 2; g >= L.g0; --g) {
    const int nx = L.nx[g], ny = L.ny[g], n = nx * ny;
    const int nxc = L.nx[g + 1], nyc = L.ny[g + 1];
    const bool wm = wmode(g);
    if (!wm && wmode(g + 1)) __syncthreads();   // results of warp 0 become visible to the block
    const int lim = wm ? 32 : (int)blockDim.x;
    const bool act = tid < lim;
    const T* st = sst + 9 * L.off[g];
    const T* dinv = sdi + L.off[g];
    const T* b = B(g);
    T* c = cur[g];
    T* o = oth[g];
    const T* xc = cur[g + 1];
    if (act)
      for (int idx = tid; idx < n; idx += lim) {
        const int y = idx / nx, x = idx - y * nx;
        c[idx] += prolong_at(x, y, nxc, nyc, xc, 1, 0);
      }
    lsync(wm);
    for (int s = 0; s < nu; ++s) {
      if (act)
        for (int idx = tid; idx < n; idx += lim) {
          const int y = idx / nx, x = idx - y * nx;
          o[idx] = c[idx] + om * dinv[idx] * (b[idx] - sdot(st + idx * 9, nx, ny, x, y, c));
        }
      lsync(wm);
      T* t = c; c = o; o = t;
    }
    cur[g] = c;
  }
  __syncthreads();
  const int n0 = L.nx[L.g0] * L.ny[L.g0];
  const T* x0 = cur[L.g0];
  for (int idx = tid; idx < n0; idx += blockDim.x) xg[idx * w + col] = x0[idx];
}

// ------------------------------------------------------------- batched CG ---

// r = src (cast), x = 0 (x has leading dimension ldx), ||b||^2 -> FIN_INIT
// (sets the loop condition)
template <typename TS, typename T>
__global__ void __launch_bounds__(1024) k_gather(int n, int w, int k, const TS* __restrict__ src, int lds, T* __restrict__ r,
                         T* __restrict__ x, int ldx, FinArgs f) {
  int col, node, nstep;
  thread_pos(w, k, col, node, nstep);
  typename Acc<T>::type acc = 0;
  for (; node < n; node += nstep) {
    const int i = node * w + col;
    const T v = (T)src[(size_t)node * lds + col];
    r[i] = v;
    x[(size_t)node * ldx + col] = T(0);
    acc += v * v;
  }
  reduce_finalize(f, acc, w, k, FIN_INIT);
}

template <typename T, typename TD>
__global__ void __launch_bounds__(1024) k_scatter(int n, int w, int k, const T* __restrict__ x, TD* __restrict__ dst, int ldd) {
  int col, node, nstep;
  thread_pos(w, k, col, node, nstep);
  for (; node < n; node += nstep) dst[(size_t)node * ldd + col] = (TD)x[(size_t)node * w + col];
}

// a . b per column -> op (used when the finest grid is inside the coarse block)
template <typename T>
__global__ void __launch_bounds__(1024) k_dot_fin(int n, int w, int k, const T* __restrict__ a, const T* __restrict__ b, FinArgs f, int op) {
  int col, node, nstep;
  thread_pos(w, k, col, node, nstep);
  typename Acc<T>::type acc = 0;
  if (!f.done[col])
    for (; node < n; node += nstep) {
      const int i = node * w + col;
      acc += a[i] * b[i];
    }
  reduce_finalize(f, acc, w, k, op);
}

// p_new = z + beta p_old (p_new = z on a column's first iteration), formed on the
// fly at the 9 neighbours; q = A_0 p_new; p_new . q -> FIN_ALPHA.
template <typename T>
__global__ void __launch_bounds__(1024) k_matvec_p(int nx, int ny, int w, int k, const T* __restrict__ st,
                                                   const T* __restrict__ z, T* pA, T* pB, T* __restrict__ q,
                                                   FinArgs f) {
  int col, node0, nstep;
  thread_pos(w, k, col, node0, nstep);
  const int par = f.ctl->it & 1;
  const T* __restrict__ pold = par ? pB : pA;
  T* __restrict__ pnew = par ? pA : pB;
  typename Acc<T>::type acc = 0;
  if (!f.done[col]) {
    const bool first = f.iters[col] == 0;
    const T bt = first ? T(0) : (sizeof(T) == 4 ? (T)f.betaf[col] : (T)f.beta[col]);
    const int n = nx * ny, rs = nx * w;
    for (NodeIter it(node0, nstep, nx); it.node < n; it.next()) {
      const int i = it.node * w + col;
      const T s = first ? stencil9(st + it.node * 9, i, rs, w, it.node, it.x, it.y, nx, ny,
                                   [&](int e, int, int, int) { return z[e]; })
                        : stencil9(st + it.node * 9, i, rs, w, it.node, it.x, it.y, nx, ny,
                                   [&](int e, int, int, int) { return z[e] + bt * pold[e]; });
      const T pi = first ? z[i] : z[i] + bt * pold[i];
      pnew[i] = pi;
      q[i] = s;
      acc += pi * s;
    }
  }
  reduce_finalize(f, acc, w, k, FIN_ALPHA);
}

// x += alpha p_new (x has leading dimension ldx); r -= alpha q; r . r -> FIN_CONV
// (sets the loop condition)
template <typename T>
__global__ void __launch_bounds__(1024) k_update_xr(int n, int w, int k, const T* pA, const T* pB, const T* __restrict__ q,
                            T* __restrict__ x, int ldx, T* __restrict__ r, FinArgs f) {
  int col, node, nstep;
  thread_pos(w, k, col, node, nstep);
  const T* __restrict__ pnew = (f.ctl->it & 1) ? pA : pB;
  typename Acc<T>::type acc = 0;
  if (!f.done[col]) {
    const T a = sizeof(T) == 4 ? (T)f.alphaf[col] : (T)f.alpha[col];
    for (; node < n; node += nstep) {
      const int i = node * w + col;
      x[(size_t)node * ldx + col] += a * pnew[i];
      const T rv = r[i] - a * q[i];
      r[i] = rv;
      acc += rv * rv;
    }
  }
  reduce_finalize(f, acc, w, k, FIN_CONV);
}

__global__ void k_clear_done(int w, int* done) {
  for (int i = threadIdx.x; i < w; i += blockDim.x) done[i] = 0;
}

// ------------------------------------------------------------ host side ---

static int alloc_block(void** p, size_t bytes) {
  SG_TRY_CUDA(cudaMalloc(p, std::max<size_t>(bytes, 16)));
  return SG_OK;
}

static void free_inner_bufs(InnerWork& iw) {
  void* bufs[] = {iw.x, iw.r, iw.z, iw.zt, iw.pA, iw.pB, iw.q, iw.part, iw.rho, iw.pq, iw.rr, iw.bb,
                  iw.alpha, iw.beta, iw.alphaf, iw.betaf, iw.done, iw.iters, iw.ctl};
  for (void* b : bufs) cudaFree(b);
  for (auto v : {&iw.cb, &iw.cx, &iw.cxt})
    for (void* b : *v) cudaFree(b);
  iw = InnerWork();
}

void free_inner_work(sg_problem* h) {
  free_inner_bufs(h->iw32);
  free_inner_bufs(h->iw64);
}

int ensure_inner_work(sg_problem* h, int dtype, int wcap) {
  if (h->grids.empty()) {
    set_error("inner solve: no multigrid hierarchy (mesh missing, not a power-of-two square, or A_0 not a 9-point operator)");
    return SG_ERR_UNSUPPORTED;
  }
  if (wcap > 1024) {
    set_error("inner solve: batch of %d columns exceeds 1024", wcap);
    return SG_ERR_UNSUPPORTED;
  }
  if ((long long)h->grids[0].n * wcap >= (1LL << 31)) {
    set_error("inner solve: n x w = %lld exceeds the 32-bit element indexing", (long long)h->grids[0].n * wcap);
    return SG_ERR_UNSUPPORTED;
  }
  InnerWork& iw = dtype == SG_F64 ? h->iw64 : h->iw32;
  if (iw.wcap >= wcap) return SG_OK;
  if (h->capturing) {
    set_error("inner solve: workspace must be allocated before graph capture");
    return SG_ERR_UNSUPPORTED;
  }
  clear_graphs(h);   // graphs hold pointers into the old workspace
  SG_TRY_CUDA(cudaDeviceSynchronize());
  free_inner_bufs(iw);
  const size_t es = dtype == SG_F64 ? 8 : 4;
  iw.esize = es;
  iw.wcap = wcap;
  const size_t nb = (size_t)h->grids[0].n * wcap * es;
  for (void** b : {&iw.x, &iw.r, &iw.z, &iw.zt, &iw.pA, &iw.pB, &iw.q}) SG_TRY(alloc_block(b, nb));
  const int G = (int)h->grids.size();
  iw.cb.assign(G, nullptr);
  iw.cx.assign(G, nullptr);
  iw.cxt.assign(G, nullptr);
  for (int g = 1; g < G; ++g) {
    const size_t bytes = (size_t)h->grids[g].n * wcap * es;
    SG_TRY(alloc_block(&iw.cb[g], bytes));
    SG_TRY(alloc_block(&iw.cx[g], bytes));
    SG_TRY(alloc_block(&iw.cxt[g], bytes));
  }
  iw.part_blocks = h->num_sms * 8;
  SG_TRY(alloc_block((void**)&iw.part, (size_t)iw.part_blocks * wcap * sizeof(double)));
  for (double** b : {&iw.rho, &iw.pq, &iw.rr, &iw.bb, &iw.alpha, &iw.beta})
    SG_TRY(alloc_block((void**)b, (size_t)wcap * sizeof(double)));
  for (float** b : {&iw.alphaf, &iw.betaf}) SG_TRY(alloc_block((void**)b, (size_t)wcap * sizeof(float)));
  SG_TRY(alloc_block((void**)&iw.done, (size_t)wcap * sizeof(int)));
  SG_TRY(alloc_block((void**)&iw.iters, (size_t)wcap * sizeof(int)));
  SG_TRY(alloc_block((void**)&iw.ctl, sizeof(InnerCtl)));
  SG_TRY_CUDA(cudaMemset(iw.ctl, 0, sizeof(InnerCtl)));
  SG_TRY_CUDA(cudaMemset(iw.done, 0, (size_t)wcap * sizeof(int)));
  SG_TRY_CUDA(cudaMemset(iw.iters, 0, (size_t)wcap * sizeof(int)));
  return SG_OK;
}

int check_prec_opts(const sg_prec_opts& o) {
  if (o.nu < 1 || o.nu > 16 || !(o.omega > 0.0) || o.inner_maxit < 1 || o.inner_fixed_iters < 0 ||
      !(o.inner_tol >= 0.0)) {
    set_error("prec opts: need 1 <= nu <= 16, omega > 0, inner_maxit >= 1, inner_tol >= 0");
    return SG_ERR_INVALID_ARG;
  }
  return SG_OK;
}

static FinArgs make_fin(sg_problem* h, InnerWork& iw, const sg_prec_opts& o) {
  FinArgs f;
  f.part = iw.part;
  f.ldp = iw.wcap;
  f.ctl = iw.ctl;
  f.rho = iw.rho; f.pq = iw.pq; f.rr = iw.rr; f.bb = iw.bb; f.alpha = iw.alpha; f.beta = iw.beta;
  f.alphaf = iw.alphaf;
  f.betaf = iw.betaf;
  f.done = iw.done;
  f.iters = iw.iters;
  f.status = h->status;
  f.tol2 = o.inner_tol * o.inner_tol;
  f.maxit = o.inner_maxit;
  f.fixed = o.inner_fixed_iters;
  f.cond = 0;
  f.has_cond = 0;
  f.flag = nullptr;
  f.iacc = h->iacc;
  return f;
}

template <typename T>
static int launch_coarse(sg_problem* h, int g0, const T* b, T* x, int w, const sg_prec_opts& o, const int* done,
                         cudaStream_t s) {
  CoarseGrids L;
  L.g0 = g0;
  L.G = (int)h->grids.size();
  int tot = 0;
  for (int g = g0; g < L.G; ++g) {
    const GridLevel& G = h->grids[g];
    L.nx[g] = G.nx;
    L.ny[g] = G.ny;
    L.off[g] = tot;
    tot += G.n;
    L.st[g] = sizeof(T) == 8 ? (const void*)G.st64 : (const void*)G.st32;
    L.dinv[g] = sizeof(T) == 8 ? (const void*)G.dinv64 : (const void*)G.dinv32;
  }
  const size_t smem = (size_t)13 * tot * sizeof(T);
  SG_TRY_CUDA(cudaFuncSetAttribute(k_vcycle_coarse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  { k_vcycle_coarse<T><<<w, 1024, smem, s>>>(L, tot, w, b, x, (T)o.omega, o.nu, done); ::sghsc::note_launch(); }
  SG_CHECK_LAUNCH();
  return SG_OK;
}

// One V-cycle on grid g applied to b (zero initial guess). *out receives the
// buffer holding the result (x or xt). With fdot (finest grid only) the last
// kernel also reduces b . result into FIN_RHO.
template <typename T>
static int vcycle(sg_problem* h, InnerWork& iw, int g, const T* b, T* x, T* xt, int w, const sg_prec_opts& o,
                  cudaStream_t s, const FinArgs* fdot, const T** out) {
  const T om = (T)o.omega;
  FinArgs fz = make_fin(h, iw, o);
  if (g >= h->cb_level) {
    SG_TRY(launch_coarse<T>(h, g, b, x, w, o, iw.done, s));
    if (fdot) {
      const Shape sh = make_shape(h, h->grids[g].n, w, 1);
      { k_dot_fin<T><<<sh.grid, sh.bdim, 0, s>>>(h->grids[g].n, w, sh.k, b, x, *fdot, FIN_RHO); ::sghsc::note_launch(); }
    }
    *out = x;
    return SG_OK;
  }
  const GridLevel& G = h->grids[g];
  const GridLevel& C = h->grids[g + 1];
  const T* st = sizeof(T) == 8 ? (const T*)G.st64 : (const T*)G.st32;
  const T* dinv = sizeof(T) == 8 ? (const T*)G.dinv64 : (const T*)G.dinv32;
  const Shape sh = make_shape(h, G.n, w);
  const Shape shd = make_shape(h, G.n, w, 1);   // kernels that end in a reduction
  const Shape shc = make_shape(h, C.n, w);
  T* cur = x;
  T* oth = xt;
  if (o.nu == 1) {
    { k_smooth0<T><<<sh.grid, sh.bdim, 0, s>>>(G.n, w, sh.k, dinv, b, cur, om, iw.done); ::sghsc::note_launch(); }
  } else {
    { k_smooth00<T><<<sh.grid, sh.bdim, 0, s>>>(G.nx, G.ny, w, sh.k, st, dinv, b, cur, om, iw.done); ::sghsc::note_launch(); }
    for (int it = 2; it < o.nu; ++it) {
      { k_jacobi<T, false><<<sh.grid, sh.bdim, 0, s>>>(G.nx, G.ny, w, sh.k, st, dinv, b, cur, oth, om, fz); ::sghsc::note_launch(); }
      std::swap(cur, oth);
    }
  }
  T* cb = (T*)iw.cb[g + 1];
  { k_resid_restrict<T><<<shc.grid, shc.bdim, 0, s>>>(G.nx, G.ny, C.nx, C.ny, w, shc.k, st, b, cur, cb, iw.done); ::sghsc::note_launch(); }
  const T* xc = nullptr;
  SG_TRY(vcycle<T>(h, iw, g + 1, cb, (T*)iw.cx[g + 1], (T*)iw.cxt[g + 1], w, o, s, nullptr, &xc));
  if (o.nu == 1 && fdot) {
    { k_prolong_jacobi<T, true><<<shd.grid, shd.bdim, 0, s>>>(G.nx, G.ny, C.nx, C.ny, w, sh.k, st, dinv, b, cur, xc, oth, om, *fdot); ::sghsc::note_launch(); }
  } else {
    { k_prolong_jacobi<T, false><<<sh.grid, sh.bdim, 0, s>>>(G.nx, G.ny, C.nx, C.ny, w, sh.k, st, dinv, b, cur, xc, oth, om, fz); ::sghsc::note_launch(); }
  }
  std::swap(cur, oth);
  for (int it = 1; it < o.nu; ++it) {
    if (it == o.nu - 1 && fdot) {
      { k_jacobi<T, true><<<shd.grid, shd.bdim, 0, s>>>(G.nx, G.ny, w, sh.k, st, dinv, b, cur, oth, om, *fdot); ::sghsc::note_launch(); }
    } else {
      { k_jacobi<T, false><<<sh.grid, sh.bdim, 0, s>>>(G.nx, G.ny, w, sh.k, st, dinv, b, cur, oth, om, fz); ::sghsc::note_launch(); }
    }
    std::swap(cur, oth);
  }
  SG_CHECK_LAUNCH();
  *out = cur;
  return SG_OK;
}

template <typename T>
static int inner_solve_t(sg_problem* h, const void* src, int ld_src, int src_t, void* dst, int ld_dst, int dst_t,
                         int w, const sg_prec_opts& o, cudaStream_t s) {
  InnerWork& iw = sizeof(T) == 8 ? h->iw64 : h->iw32;
  const GridLevel& G = h->grids[0];
  const Shape sh = make_shape(h, G.n, w, 1);    // gather / matvec / update end in reductions
  const Shape shs = make_shape(h, G.n, w);
  T* x = (T*)iw.x;
  T* r = (T*)iw.r;
  T* q = (T*)iw.q;
  T* pA = (T*)iw.pA;
  T* pB = (T*)iw.pB;
  const T* st = sizeof(T) == 8 ? (const T*)G.st64 : (const T*)G.st32;
  FinArgs fa = make_fin(h, iw, o);
  // the iterate lives in the destination itself when the element types agree
  const bool direct = dst_t == (sizeof(T) == 8 ? SG_F64 : SG_F32);
  T* xd = direct ? (T*)dst : x;
  const int ldx = direct ? ld_dst : w;
  auto pre = [&](cudaStream_t ps, const LoopCtl& lc) -> int {
    FinArgs f = fa;
    f.cond = lc.cond;
    f.has_cond = lc.has_cond;
    f.flag = lc.flag;
    if (src_t == SG_F64)
      { k_gather<double, T><<<sh.grid, sh.bdim, 0, ps>>>(G.n, w, sh.k, (const double*)src, ld_src, r, xd, ldx, f); ::sghsc::note_launch(); }
    else
      { k_gather<float, T><<<sh.grid, sh.bdim, 0, ps>>>(G.n, w, sh.k, (const float*)src, ld_src, r, xd, ldx, f); ::sghsc::note_launch(); }
    SG_CHECK_LAUNCH();
    return SG_OK;
  };
  auto body = [&](cudaStream_t bs, const LoopCtl& lc) -> int {
    FinArgs f = fa;
    f.cond = lc.cond;
    f.has_cond = lc.has_cond;
    f.flag = lc.flag;
    const T* z = nullptr;
    SG_TRY(vcycle<T>(h, iw, 0, r, (T*)iw.z, (T*)iw.zt, w, o, bs, &f, &z));
    { k_matvec_p<T><<<sh.grid, sh.bdim, 0, bs>>>(G.nx, G.ny, w, sh.k, st, z, pA, pB, q, f); ::sghsc::note_launch(); }
    { k_update_xr<T><<<sh.grid, sh.bdim, 0, bs>>>(G.n, w, sh.k, pA, pB, q, xd, ldx, r, f); ::sghsc::note_launch(); }
    SG_CHECK_LAUNCH();
    return SG_OK;
  };
  SG_TRY(capture_while(h, s, pre, body));
  if (!direct) {
    if (dst_t == SG_F64)
      { k_scatter<T, double><<<shs.grid, shs.bdim, 0, s>>>(G.n, w, shs.k, x, (double*)dst, ld_dst); ::sghsc::note_launch(); }
    else
      { k_scatter<T, float><<<shs.grid, shs.bdim, 0, s>>>(G.n, w, shs.k, x, (float*)dst, ld_dst); ::sghsc::note_launch(); }
    SG_CHECK_LAUNCH();
  }
  return SG_OK;
}

int inner_solve(sg_problem* h, int dtype, const void* src, int ld_src, int src_t, void* dst, int ld_dst, int dst_t,
                int w, const sg_prec_opts& o, cudaStream_t s) {
  SG_TRY(check_prec_opts(o));
  if (w <= 0) return SG_OK;
  SG_TRY(ensure_inner_work(h, dtype, std::max(w, h->wmax)));
  if (dtype == SG_F64) return inner_solve_t<double>(h, src, ld_src, src_t, dst, ld_dst, dst_t, w, o, s);
  return inner_solve_t<float>(h, src, ld_src, src_t, dst, ld_dst, dst_t, w, o, s);
}

int inner_vcycle(sg_problem* h, int dtype, const void* B, void* X, int w, const sg_prec_opts& o, cudaStream_t s) {
  SG_TRY(check_prec_opts(o));
  SG_TRY(ensure_inner_work(h, dtype, std::max(w, h->wmax)));
  const size_t es = dtype == SG_F64 ? 8 : 4;
  InnerWork& iw = dtype == SG_F64 ? h->iw64 : h->iw32;
  { k_clear_done<<<1, 1024, 0, s>>>(w, iw.done); ::sghsc::note_launch(); }
  const void* res = nullptr;
  if (dtype == SG_F64) {
    const double* r = nullptr;
    SG_TRY(vcycle<double>(h, iw, 0, (const double*)B, (double*)iw.z, (double*)iw.zt, w, o, s, nullptr, &r));
    res = r;
  } else {
    const float* r = nullptr;
    SG_TRY(vcycle<float>(h, iw, 0, (const float*)B, (float*)iw.z, (float*)iw.zt, w, o, s, nullptr, &r));
    res = r;
  }
  SG_CHECK_LAUNCH();
  SG_TRY_CUDA(cudaMemcpyAsync(X, res, (size_t)h->grids[0].n * w * es, cudaMemcpyDeviceToDevice, s));
  return SG_OK;
}

// ---------------------------------------------------------------------------
// V-cycle without allocation (sg_vcycle_apply_static).
//
// For callers that must not allocate device memory while they run -- code
// that executes inside a stream capture, an allocator or memory-pool hook,
// or a process whose device memory is budgeted and already handed out. The
// level buffers of the V-cycle live in this file-scope array instead of the
// handle's workspace. Every GPU that loads the library holds the array until
// the process exits; all calls on one device share it and it keeps the
// contents of the last call, so calls whose GPU work overlaps (other streams,
// other threads) race.
// ---------------------------------------------------------------------------

constexpr size_t STATIC_SCRATCH_BYTES = (size_t)32 << 20;
static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

constexpr int STATIC_MAX_DEVICES = 64;
static void* g_static_scratch_ptr[STATIC_MAX_DEVICES];
static cudaError_t g_static_scratch_err[STATIC_MAX_DEVICES];
static std::once_flag g_static_scratch_once[STATIC_MAX_DEVICES];

// Device address of g_static_scratch on the current device; resolved once per
// device (the name is only a host-side stand-in for the device array).
static int static_scratch(void** out) {
  int dev = 0;
  SG_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= STATIC_MAX_DEVICES) {
    set_error("sg_vcycle_apply_static: device ordinal %d not supported", dev);
    return SG_ERR_UNSUPPORTED;
  }
  std::call_once(g_static_scratch_once[dev], [dev]() {
    g_static_scratch_err[dev] = cudaGetSymbolAddress(&g_static_scratch_ptr[dev], g_static_scratch);
  });
  SG_TRY_CUDA(g_static_scratch_err[dev]);
  *out = g_static_scratch_ptr[dev];
  return SG_OK;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Bytes of V-cycle scratch for w columns: the done mask, two iterates on the
// finest grid and three blocks per coarser grid.
static size_t static_vcycle_bytes(const sg_problem* h, int w, size_t es) {
  size_t b = align256((size_t)w * sizeof(int));
  b += 2 * align256((size_t)h->grids[0].n * w * es);
  for (size_t g = 1; g < h->grids.size(); ++g) b += 3 * align256((size_t)h->grids[g].n * w * es);
  return b;
}

int vcycle_static(sg_problem* h, int dtype, const void* B, void* X, int w, const sg_prec_opts& o, cudaStream_t s) {
  SG_TRY(check_prec_opts(o));
  if (h->grids.empty()) {
    set_error("sg_vcycle_apply_static: no multigrid hierarchy (mesh missing or not a power-of-two square)");
    return SG_ERR_UNSUPPORTED;
  }
  const size_t es = dtype == SG_F64 ? 8 : 4;
  const size_t need = static_vcycle_bytes(h, w, es);
  if (need > STATIC_SCRATCH_BYTES) {
    set_error("sg_vcycle_apply_static: %d columns of %d nodes need %zu bytes of scratch, above the fixed %zu",
              w, h->grids[0].n, need, STATIC_SCRATCH_BYTES);
    return SG_ERR_INVALID_ARG;
  }
  void* base = nullptr;
  SG_TRY(static_scratch(&base));
  unsigned char* p = (unsigned char*)base;
  InnerWork sw;  // views into the static array; nothing here allocates
  sw.wcap = w;
  sw.esize = es;
  sw.done = (int*)p;
  p += align256((size_t)w * sizeof(int));
  sw.z = p;
  p += align256((size_t)h->grids[0].n * w * es);
  sw.zt = p;
  p += align256((size_t)h->grids[0].n * w * es);
  const int G = (int)h->grids.size();
  sw.cb.assign(G, nullptr);
  sw.cx.assign(G, nullptr);
  sw.cxt.assign(G, nullptr);
  for (int g = 1; g < G; ++g) {
    const size_t bytes = align256((size_t)h->grids[g].n * w * es);
    sw.cb[g] = p;
    p += bytes;
    sw.cx[g] = p;
    p += bytes;
    sw.cxt[g] = p;
    p += bytes;
  }
  // the kernels skip columns whose done flag is set: start from all zero
  SG_TRY_CUDA(cudaMemsetAsync(sw.done, 0, (size_t)w * sizeof(int), s));
  const void* res = nullptr;
  if (dtype == SG_F64) {
    const double* r = nullptr;
    SG_TRY(vcycle<double>(h, sw, 0, (const double*)B, (double*)sw.z, (double*)sw.zt, w, o, s, nullptr, &r));
    res = r;
  } else {
    const float* r = nullptr;
    SG_TRY(vcycle<float>(h, sw, 0, (const float*)B, (float*)sw.z, (float*)sw.zt, w, o, s, nullptr, &r));
    res = r;
  }
  SG_CHECK_LAUNCH();
  SG_TRY_CUDA(cudaMemcpyAsync(X, res, (size_t)h->grids[0].n * w * es, cudaMemcpyDeviceToDevice, s));
  return SG_OK;
}

}  // namespace sghsc

extern "C" int sg_vcycle_apply_static(sg_problem* h, const void* B, void* X, int w, int dtype,
                                      const sg_prec_opts* opts, void* stream) {
  sghsc::set_error("");
  if (!h || !B || !X || !opts || w <= 0 || w > 1024 || (dtype != SG_F64 && dtype != SG_F32)) {
    sghsc::set_error("sg_vcycle_apply_static: invalid arguments");
    return SG_ERR_INVALID_ARG;
  }
  return sghsc::vcycle_static(h, dtype, B, X, w, *opts, (cudaStream_t)stream);
}
