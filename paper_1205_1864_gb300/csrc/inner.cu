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
// Thread mapping: the blocks of a batch have a padded width wp (a multiple of
// N = 16 bytes / element size); a thread owns a column group of N adjacent
// columns, moved with 16-byte loads and stores. A block has k*ng threads
// (ng = wp/N groups, k = max(1, 1024 / ng)), thread t always handles group
// t mod ng and node t / ng of each block pass (pointwise kernels: passes in
// grid-stride order; stencil kernels: down a column strip, StripIter), so
// per-column partial sums are register accumulations followed by a fixed-order
// block reduction; the last block to finish a reduction kernel
// sums the block partials in block order and updates the CG scalars, so the
// results do not depend on scheduling and no separate finalisation launch is
// needed. The iteration loop is a CUDA graph WHILE node whose condition the
// convergence kernel sets (graph.cu).
//
// V-cycle kernels (weighted Jacobi, nu sweeps before and after, bilinear
// transfers, Galerkin coarse operators built in setup.cu):
//   k_smooth00        two sweeps from a zero iterate in one pass
//   k_resid_restrict_t  the residual b - A x formed once per fine node in shared
//                     memory (tiles of coarse nodes) and restricted
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
#include "vec.cuh"

namespace sghsc {

constexpr int MAX_LEVELS = 16;

// Column groups: the batch buffers are node-major with a padded width wp (a
// multiple of N = 16 bytes / sizeof(T)), and each thread owns N adjacent
// columns of a node, moved with one 16-byte load or store. Per-node data
// (stencil, inverse diagonal, grid position) is then read once per N columns
// and the address arithmetic is shared by N elements.
template <typename T>
struct VW;
template <>
struct VW<float> {
  using type = float4;
  static constexpr int N = 4;
};
template <>
struct VW<double> {
  using type = double2;
  static constexpr int N = 2;
};

template <typename T>
struct Vec {
  static constexpr int N = VW<T>::N;
  T a[N];
};

template <typename T>
__device__ __forceinline__ Vec<T> vld(const T* p) {
  const typename VW<T>::type v = *reinterpret_cast<const typename VW<T>::type*>(p);
  Vec<T> r;
  if constexpr (VW<T>::N == 4) {
    r.a[0] = v.x; r.a[1] = v.y; r.a[2] = v.z; r.a[3] = v.w;
  } else {
    r.a[0] = v.x; r.a[1] = v.y;
  }
  return r;
}

template <typename T>
__device__ __forceinline__ void vst(T* p, const Vec<T>& r) {
  typename VW<T>::type v;
  if constexpr (VW<T>::N == 4) {
    v.x = r.a[0]; v.y = r.a[1]; v.z = r.a[2]; v.w = r.a[3];
  } else {
    v.x = r.a[0]; v.y = r.a[1];
  }
  *reinterpret_cast<typename VW<T>::type*>(p) = v;
}

template <typename T>
__device__ __forceinline__ Vec<T> vzero() {
  Vec<T> r;
#pragma unroll
  for (int u = 0; u < VW<T>::N; ++u) r.a[u] = T(0);
  return r;
}

// bit u set when column c0 + u is finished
template <int N>
__device__ __forceinline__ unsigned done_mask(const int* __restrict__ done, int c0) {
  unsigned m = 0;
#pragma unroll
  for (int u = 0; u < N; ++u) m |= (done[c0 + u] ? 1u : 0u) << u;
  return m;
}

struct Shape {
  int ng, k, bdim, grid;
};

// ng column groups per node, k = max(1, 1024 / ng) nodes per block pass,
// at most `per_sm` blocks per SM. The reduction kernels use one block per SM:
// few block partials per column, so the last-block reduction stays short.
static Shape make_shape(const sg_problem* h, int nodes, int ng, int per_sm = 2) {
  Shape s;
  s.ng = ng;
  s.k = std::max(1, 1024 / ng);
  s.bdim = s.k * ng;
  s.grid = std::max(1, std::min(ceil_div(nodes, s.k), h->num_sms * per_sm));
  return s;
}

// The grid of s clamped to what can be resident at once for kernel kern (its
// register and shared-memory use), so no launch runs in two waves.
template <typename K>
static Shape fit(const sg_problem* h, Shape s, K kern) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, s.bdim, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  s.grid = std::max(1, std::min(s.grid, h->num_sms * per_sm));
  return s;
}

template <typename T>
static int padded_width(int w) {
  constexpr int N = 16 / (int)sizeof(T);
  return (w + N - 1) / N * N;
}

enum { FIN_INIT = 0, FIN_RHO = 1, FIN_ALPHA = 2, FIN_CONV = 3 };

// Per-column CG state (global memory; the last block of each reduction
// updates it) and the reduction target.
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
  int count_iacc;   // this block adds finished columns to iacc
};

// The blocks doing one phase: this block's index and their number.
struct Blk {
  int bid, nb;
};

__device__ __forceinline__ Blk this_grid() { return Blk{(int)blockIdx.x, (int)gridDim.x}; }

// Thread t of a block: column group t mod ng, node slice t / ng; false for
// threads past k*ng (blocks wider than the phase needs).
__device__ __forceinline__ bool thread_pos(int ng, int k, Blk B, int& cg, int& node0, int& nstep) {
  if ((int)threadIdx.x >= k * ng) return false;
  cg = threadIdx.x % ng;
  node0 = B.bid * k + threadIdx.x / ng;
  nstep = B.nb * k;
  return true;
}

// Lanes of this thread's warp that exist (the last warp of a block whose size
// is not a multiple of 32 is partial).
__device__ __forceinline__ unsigned warp_lanes() {
  const unsigned left = blockDim.x - (threadIdx.x & ~31u);
  return left >= 32 ? 0xffffffffu : ((1u << left) - 1u);
}

// Largest power of two g <= 32 with g * cols <= blockDim (at least 1): the
// lanes that reduce one column, so one pass covers as many columns as fit.
__device__ __forceinline__ int group_lanes(int cols) {
  int g = 1;
  while (g < 32 && 2 * g * cols <= (int)blockDim.x) g *= 2;
  return g;
}

template <typename A>
__device__ __forceinline__ A group_shfl_sum(A s, int g) {
  const unsigned m = warp_lanes();
  for (int o = g >> 1; o > 0; o >>= 1) s += __shfl_down_sync(m, s, o, g);
  return s;
}

// Per-column block partial: thread (slice, cg) holds columns cg*N .. cg*N+N-1;
// the k slices of each column are summed in the accumulation type A in a fixed
// order and stored at part[bid][c] (leading dimension ldp).
template <typename A, int N>
__device__ __forceinline__ void block_col_reduce(const A (&v)[N], int wp, int k, A* part, int ldp, int bid) {
  __shared__ A red[4096 / (sizeof(A) / 4)];   // k * wp <= 1024 * N elements
  const int ng = wp / N;
  if ((int)threadIdx.x < k * ng) {
    const int cg = threadIdx.x % ng, slice = threadIdx.x / ng;
#pragma unroll
    for (int u = 0; u < N; ++u) red[slice * wp + cg * N + u] = v[u];
  }
  __syncthreads();
  const int g = group_lanes(wp);
  const int per_pass = blockDim.x / g;
  const int lane = threadIdx.x % g;
  for (int c0 = 0; c0 < wp; c0 += per_pass) {
    const int c = c0 + (int)threadIdx.x / g;
    A s = A(0);
    if (c < wp)
      for (int j = lane; j < k; j += g) s += red[j * wp + c];
    s = group_shfl_sum(s, g);
    if (c < wp && lane == 0) {
      part[(size_t)bid * ldp + c] = s;
      __threadfence();  // only the writers of partials need the release fence
    }
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

// Column totals of the block partials into colsum[0..wp). Column c is summed
// by a lane group in the accumulation type A (blocks lane, lane + g, ...
// loaded 16 at a time, then the g-wide shuffle): a fixed order, so every
// caller gets the same bits. Ends with a block barrier.
template <typename A>
__device__ void col_totals(const A* part, int ldp, int nblk, int wp, double* colsum) {
  const int g = group_lanes(wp);
  const int per_pass = blockDim.x / g;
  const int lane = threadIdx.x % g;
  for (int c0 = 0; c0 < wp; c0 += per_pass) {
    const int gc = c0 + (int)threadIdx.x / g;
    A s = A(0);
    if (gc < wp) {
      constexpr int B = 16;
      for (int b0 = lane; b0 < nblk; b0 += B * g) {
        A v[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
          const int b = b0 + u * g;
          v[u] = b < nblk ? __ldcg(&part[(size_t)b * ldp + gc]) : A(0);
        }
#pragma unroll
        for (int u = 0; u < B; ++u) s += v[u];
      }
    }
    s = group_shfl_sum(s, g);
    if (gc < wp && lane == 0) colsum[gc] = (double)s;
  }
  __syncthreads();
}

// The CG scalar updates of every column from its total colsum[c], done by
// threads 0..wp-1 in FP64 (so only the first ceil(wp/32) warps issue FP64
// work); *cnt (zeroed by the caller before a barrier) counts the columns left.
__device__ void col_update(const FinArgs& f, int op, int wp, const double* colsum, int* cnt) {
  for (int c = threadIdx.x; c < wp; c += blockDim.x) {
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
        if (fin && f.count_iacc) {
          atomicAdd((unsigned long long*)&f.iacc[0], (unsigned long long)it);
          atomicMax(&f.iacc[1], (long long)it);
        }
      }
    }
    if (!f.done[c]) atomicAdd(cnt, 1);
  }
}

// Last block of a stand-alone reduction kernel: totals, scalar updates, the
// iteration counter and the loop condition of the graph WHILE node.
template <typename A>
__device__ void fin_columns(const FinArgs& f, int op, int wp, int nblk) {
  __shared__ int cnt;
  __shared__ double colsum[1024];
  if (threadIdx.x == 0) cnt = 0;
  col_totals<A>((const A*)f.part, f.ldp, nblk, wp, colsum);
  col_update(f, op, wp, colsum, &cnt);
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

template <typename A, int N>
__device__ __forceinline__ void reduce_finalize(const FinArgs& f, const A (&v)[N], int wp, int k, int op) {
  block_col_reduce<A, N>(v, wp, k, (A*)f.part, f.ldp, blockIdx.x);
  if (last_block(&f.ctl->ticket)) fin_columns<A>(f, op, wp, gridDim.x);
}

// (P xc) at fine node (fx, fy): bilinear interpolation from the coarse grid,
// coarse node (X, Y) sitting on fine node (2X+1, 2Y+1), zero outside
// (one column, used by the coarse-grid phase).
template <typename T>
__device__ __forceinline__ T prolong_at(int fx, int fy, int nxc, int nyc, const T* __restrict__ xc) {
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
      acc += wy[iy] * wx[ix] * xc[Ys[iy] * nxc + Xs[ix]];
    }
  }
  return acc;
}

// Node order of the 9-point stencil phases. The grid is cut into column strips
// k nodes wide (the nodes of one block pass); the (strip, row) units are split
// into one contiguous share per block, and a block walks its share row by row
// down a strip, so the rows y - 1 and y that the stencils of row y + 1 read are
// still in L1 from the two passes before (a grid-stride order along x would
// fetch every row three times from L2, once per neighbouring row). lx: this
// thread's node within the pass.
struct StripIter {
  int x, y, node, u, u1, cx, lx, k, nx, ny;
  __device__ __forceinline__ StripIter(Blk B, int lx_, int k_, int nx_, int ny_)
      : lx(lx_), k(k_), nx(nx_), ny(ny_) {
    const long long tot = (long long)((nx + k - 1) / k) * ny;
    u = (int)(tot * B.bid / B.nb);
    u1 = (int)(tot * (B.bid + 1) / B.nb);
    cx = u / ny;
    y = u - cx * ny;
    x = cx * k + lx;
    node = y * nx + x;
  }
  __device__ __forceinline__ bool valid() const { return u < u1; }
  __device__ __forceinline__ bool inside() const { return x < nx; }
  __device__ __forceinline__ void next() {
    ++u;
    if (++y == ny) {
      y = 0;
      ++cx;
      x = cx * k + lx;
    }
    node = y * nx + x;
  }
};

// Thread t of a block in the stencil phases: column group t mod ng, node t / ng
// of each pass; false for threads past k*ng.
__device__ __forceinline__ bool strip_pos(int ng, int k, int& cg, int& lx) {
  if ((int)threadIdx.x >= k * ng) return false;
  cg = threadIdx.x % ng;
  lx = threadIdx.x / ng;
  return true;
}

// sum_j a_ij val(e_j, j) over the 9-point stencil of node (x, y) for the N
// columns of a group; e_j = i + dy*rs + dx*wp is the element index of the
// group at neighbour j = node + dy*nx + dx (rs = nx*wp). Interior nodes take a
// branch-free path.
template <typename T, typename F>
__device__ __forceinline__ Vec<T> stencil9(const T* __restrict__ s9, int i, int rs, int wp, int node, int x, int y,
                                           int nx, int ny, F val) {
  constexpr int N = VW<T>::N;
  Vec<T> acc = vzero<T>();
  if (x > 0 && x < nx - 1 && y > 0 && y < ny - 1) {
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const T a = s9[(dy + 1) * 3 + (dx + 1)];
        const Vec<T> v = val(i + dy * rs + dx * wp, node + dy * nx + dx);
#pragma unroll
        for (int u = 0; u < N; ++u) acc.a[u] += a * v.a[u];
      }
    return acc;
  }
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
    if (y + dy < 0 || y + dy >= ny) continue;
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      if (x + dx < 0 || x + dx >= nx) continue;
      const T a = s9[(dy + 1) * 3 + (dx + 1)];
      const Vec<T> v = val(i + dy * rs + dx * wp, node + dy * nx + dx);
#pragma unroll
      for (int u = 0; u < N; ++u) acc.a[u] += a * v.a[u];
    }
  }
  return acc;
}

// ---------------------------------------------------------------- phases ---
// Each phase is the body of one stand-alone kernel, over the blocks B; the
// reduction phases return the thread's per-column partial sums in acc.

// one sweep from zero: x = omega D^{-1} b
template <typename T>
__device__ __forceinline__ void ph_smooth0(Blk B, int n, int wp, int k, const T* __restrict__ dinv,
                                           const T* __restrict__ b, T* __restrict__ x, T om,
                                           const int* __restrict__ done) {
  constexpr int N = VW<T>::N;
  int cg, node, nstep;
  if (!thread_pos(wp / N, k, B, cg, node, nstep)) return;
  const int c0 = cg * N;
  if (done_mask<N>(done, c0) == (1u << N) - 1) return;
  for (; node < n; node += nstep) {
    const int i = node * wp + c0;
    const T d = om * dinv[node];
    const Vec<T> bv = vld(b + i);
    Vec<T> xv;
#pragma unroll
    for (int u = 0; u < N; ++u) xv.a[u] = d * bv.a[u];
    vst(x + i, xv);
  }
}

// two sweeps from zero: x1 = omega D^{-1} b, x2 = x1 + omega D^{-1} (b - A x1)
template <typename T>
__device__ __forceinline__ void ph_smooth00(Blk B, int nx, int ny, int wp, int k, const T* __restrict__ st,
                                            const T* __restrict__ dinv, const T* __restrict__ b,
                                            T* __restrict__ x, T om, const int* __restrict__ done) {
  constexpr int N = VW<T>::N;
  int cg, lx;
  if (!strip_pos(wp / N, k, cg, lx)) return;
  const int c0 = cg * N;
  if (done_mask<N>(done, c0) == (1u << N) - 1) return;
  const int rs = nx * wp;
  for (StripIter it(B, lx, k, nx, ny); it.valid(); it.next()) {
    if (!it.inside()) continue;
    const int i = it.node * wp + c0;
    const Vec<T> ax1 = stencil9(st + it.node * 9, i, rs, wp, it.node, it.x, it.y, nx, ny, [&](int e, int j) {
      const T d = dinv[j];
      Vec<T> v = vld(b + e);
#pragma unroll
      for (int u = 0; u < N; ++u) v.a[u] *= d;
      return v;
    });
    const Vec<T> bv = vld(b + i);
    const T di = om * dinv[it.node];
    Vec<T> xv;
#pragma unroll
    for (int u = 0; u < N; ++u) xv.a[u] = di * bv.a[u] + di * (bv.a[u] - om * ax1.a[u]);
    vst(x + i, xv);
  }
}

// xo = xi + omega D^{-1} (b - A xi); with DOT also the partials of b . xo
template <typename T, bool DOT>
__device__ __forceinline__ void ph_jacobi(Blk B, int nx, int ny, int wp, int k, const T* __restrict__ st,
                                          const T* __restrict__ dinv, const T* __restrict__ b,
                                          const T* __restrict__ xi, T* __restrict__ xo, T om,
                                          const int* __restrict__ done, T (&acc)[VW<T>::N]) {
  constexpr int N = VW<T>::N;
#pragma unroll
  for (int u = 0; u < N; ++u) acc[u] = T(0);
  int cg, lx;
  if (!strip_pos(wp / N, k, cg, lx)) return;
  const int c0 = cg * N;
  if (done_mask<N>(done, c0) == (1u << N) - 1) return;
  const int rs = nx * wp;
  for (StripIter it(B, lx, k, nx, ny); it.valid(); it.next()) {
    if (!it.inside()) continue;
    const int i = it.node * wp + c0;
    const Vec<T> ax = stencil9(st + it.node * 9, i, rs, wp, it.node, it.x, it.y, nx, ny,
                               [&](int e, int) { return vld(xi + e); });
    const Vec<T> bv = vld(b + i), xv = vld(xi + i);
    const T d = om * dinv[it.node];
    Vec<T> v;
#pragma unroll
    for (int u = 0; u < N; ++u) {
      v.a[u] = xv.a[u] + d * (bv.a[u] - ax.a[u]);
      if (DOT) acc[u] += bv.a[u] * v.a[u];
    }
    vst(xo + i, v);
  }
}

// bc = P^T (b - A x), tiled: a block owns a TC x TC tile of coarse nodes. Its
// threads first form the fine residuals b - A x of the tile's (2TC+1)^2 fine
// footprint once each, for every column group, into shared memory (res); each
// coarse node then sums its 3x3 weighted fine residuals from there. The blocks
// stride over the tiles.
template <typename T>
__device__ __forceinline__ void ph_resid_restrict(Blk B, int nxf, int nyf, int nxc, int nyc, int wp, int TC,
                                                  const T* __restrict__ st, const T* __restrict__ b,
                                                  const T* __restrict__ x, T* __restrict__ bc,
                                                  const int* __restrict__ done, unsigned char* smem) {
  constexpr int N = VW<T>::N;
  using V = typename VW<T>::type;
  V* res = reinterpret_cast<V*>(smem);   // [fine footprint node][column group]
  const int ng = wp / N;
  const int ntx = (nxc + TC - 1) / TC, nty = (nyc + TC - 1) / TC;
  const int FW = 2 * TC + 1;
  const int rsf = nxf * wp;
  for (int t = B.bid; t < ntx * nty; t += B.nb) {
    const int X0 = (t % ntx) * TC, Y0 = (t / ntx) * TC;
    const int fx0 = 2 * X0, fy0 = 2 * Y0;
    for (int idx = threadIdx.x; idx < FW * FW * ng; idx += blockDim.x) {
      const int cg = idx % ng, fl = idx / ng;
      const int fx = fx0 + fl % FW, fy = fy0 + fl / FW;
      Vec<T> r = vzero<T>();
      if (fx < nxf && fy < nyf && done_mask<N>(done, cg * N) != (1u << N) - 1) {
        const int fn = fy * nxf + fx, fi = fn * wp + cg * N;
        const Vec<T> ax = stencil9(st + fn * 9, fi, rsf, wp, fn, fx, fy, nxf, nyf,
                                   [&](int e, int) { return vld(x + e); });
        const Vec<T> bv = vld(b + fi);
#pragma unroll
        for (int u = 0; u < N; ++u) r.a[u] = bv.a[u] - ax.a[u];
      }
      vst(reinterpret_cast<T*>(res + idx), r);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < TC * TC * ng; idx += blockDim.x) {
      const int cg = idx % ng, cl = idx / ng;
      const int lx = cl % TC, ly = cl / TC;
      const int X = X0 + lx, Y = Y0 + ly;
      if (X < nxc && Y < nyc) {
        Vec<T> acc = vzero<T>();
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
          const T wy = dy == 0 ? T(1) : T(0.5);
#pragma unroll
          for (int dx = -1; dx <= 1; ++dx) {
            const T wgt = (dx == 0 ? T(1) : T(0.5)) * wy;
            const int fl = (2 * ly + 1 + dy) * FW + (2 * lx + 1 + dx);
            const Vec<T> r = vld(reinterpret_cast<const T*>(res + fl * ng + cg));
#pragma unroll
            for (int u = 0; u < N; ++u) acc.a[u] += wgt * r.a[u];
          }
        }
        vst(bc + (Y * nxc + X) * wp + cg * N, acc);
      }
    }
    __syncthreads();
  }
}

// x' = x + P xc (on the fly), xo = x' + omega D^{-1} (b - A x'); DOT as ph_jacobi.
// The coarse values that the 3x3 fine neighbourhood of node (x, y) interpolates
// from lie in the 3x3 coarse patch cp[a][c], X = Xb - 1 + c, Xb = floor((x-1)/2)
// (same in y). Interpolation is separable: fine offset dx in {-1, 0, 1} takes
// the patch columns with weights Wx[dx][c], by the parity of x
//   odd x:  (1/2, 1/2, 0), (0, 1, 0), (0, 1/2, 1/2)
//   even x: (0, 1, 0), (0, 1/2, 1/2), (0, 0, 1)
// so A (P xc) at the node is sum_{a,c} K[a][c] cp[a][c] with the per-node
// weights K = Wy^T S Wx (S the 3x3 stencil, zero outside the grid), shared by
// all columns, and (P xc) at the node itself uses Wy[0] (x) Wx[0] (centre rows).
template <typename T, bool DOT>
__device__ __forceinline__ void ph_prolong_jacobi(Blk B, int nxf, int nyf, int nxc, int nyc, int wp, int k,
                                                  const T* __restrict__ st, const T* __restrict__ dinv,
                                                  const T* __restrict__ b, const T* __restrict__ x,
                                                  const T* __restrict__ xc, T* __restrict__ xo, T om,
                                                  const int* __restrict__ done, T (&acc)[VW<T>::N]) {
  constexpr int N = VW<T>::N;
#pragma unroll
  for (int u = 0; u < N; ++u) acc[u] = T(0);
  int cg, lx;
  if (!strip_pos(wp / N, k, cg, lx)) return;
  const int c0 = cg * N;
  if (done_mask<N>(done, c0) == (1u << N) - 1) return;
  const int rs = nxf * wp;
  const T h = T(0.5);
  for (StripIter it(B, lx, k, nxf, nyf); it.valid(); it.next()) {
    if (!it.inside()) continue;
    const T* s9 = st + it.node * 9;
    // separable interpolation weights by parity (rows: offset -1, 0, +1; columns: patch 0..2)
    T wxm[3][3], wym[3][3];
    const bool ox = it.x & 1, oy = it.y & 1;
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int c = 0; c < 3; ++c) { wxm[d][c] = T(0); wym[d][c] = T(0); }
    if (ox) { wxm[0][0] = h; wxm[0][1] = h; wxm[1][1] = T(1); wxm[2][1] = h; wxm[2][2] = h; }
    else { wxm[0][1] = T(1); wxm[1][1] = h; wxm[1][2] = h; wxm[2][2] = T(1); }
    if (oy) { wym[0][0] = h; wym[0][1] = h; wym[1][1] = T(1); wym[2][1] = h; wym[2][2] = h; }
    else { wym[0][1] = T(1); wym[1][1] = h; wym[1][2] = h; wym[2][2] = T(1); }
    // S masked to the grid, T1 = S Wx, K = Wy^T T1
    T t1[3][3];
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
      const bool iny = it.y + dy - 1 >= 0 && it.y + dy - 1 < nyf;
      T srow[3];
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        const bool inx = it.x + dx - 1 >= 0 && it.x + dx - 1 < nxf;
        srow[dx] = (iny && inx) ? s9[dy * 3 + dx] : T(0);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) t1[dy][c] = srow[0] * wxm[0][c] + srow[1] * wxm[1][c] + srow[2] * wxm[2][c];
    }
    T K[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) K[a][c] = wym[0][a] * t1[0][c] + wym[1][a] * t1[1][c] + wym[2][a] * t1[2][c];
    const int Xb = (it.x - 1) >> 1, Yb = (it.y - 1) >> 1;
    Vec<T> apc = vzero<T>(), pc = vzero<T>();
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int Y = Yb - 1 + a;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int X = Xb - 1 + c;
        if (Y >= 0 && Y < nyc && X >= 0 && X < nxc) {
          const Vec<T> v = vld(xc + (Y * nxc + X) * wp + c0);
          const T wc = wym[1][a] * wxm[1][c];
#pragma unroll
          for (int u = 0; u < N; ++u) {
            apc.a[u] += K[a][c] * v.a[u];
            pc.a[u] += wc * v.a[u];
          }
        }
      }
    }
    const int i = it.node * wp + c0;
    const Vec<T> ax = stencil9(s9, i, rs, wp, it.node, it.x, it.y, nxf, nyf,
                               [&](int e, int) { return vld(x + e); });
    const Vec<T> bv = vld(b + i), xv = vld(x + i);
    const T d = om * dinv[it.node];
    Vec<T> v;
#pragma unroll
    for (int u = 0; u < N; ++u) {
      v.a[u] = (xv.a[u] + pc.a[u]) + d * (bv.a[u] - (ax.a[u] + apc.a[u]));
      if (DOT) acc[u] += bv.a[u] * v.a[u];
    }
    vst(xo + i, v);
  }
}

struct CoarseGrids {
  int g0, G;
  int nx[MAX_LEVELS], ny[MAX_LEVELS], off[MAX_LEVELS];
  const void* st[MAX_LEVELS];
  const void* dinv[MAX_LEVELS];
};

template <typename T>
__device__ __forceinline__ void stage_async(T* __restrict__ dst, const T* __restrict__ src, int count) {
  for (int idx = threadIdx.x; idx < count; idx += blockDim.x) cp_async_elem(dst + idx, src + idx);
}

// Shared memory of the coarse-grid phase: per grid a right-hand side, an
// iterate and a ping-pong buffer, plus the stencils and inverse diagonals.
template <typename T>
static size_t coarse_smem_bytes(int tot) {
  return (size_t)13 * tot * sizeof(T);
}

// The V-cycle from grid g0 down, one column at a time per block (the blocks
// stride over the columns; the coarse grids are latency-bound, so the work
// spreads over as many SMs as there are columns), entirely in shared memory.
// Every coarse stencil and inverse diagonal is staged once per block, with the
// first column's right-hand side, by asynchronous copies all in flight
// together. Grids of at most 64 nodes are run by warp 0 alone with warp-level
// synchronisation. blockDim must be 1024.
template <typename T>
__device__ void ph_coarse(Blk Bk, const CoarseGrids& L, int tot, int wp, const T* __restrict__ bg,
                          T* __restrict__ xg, T om, int nu, const int* __restrict__ done, unsigned char* smem) {
  T* sm = reinterpret_cast<T*>(smem);
  T* sst = sm + 3 * tot;          // stencils [node][9] of all coarse grids
  T* sdi = sst + 9 * tot;         // inverse diagonals
  auto stg = [&](int g) { return (const T*)(sst + 9 * L.off[g]); };
  auto dig = [&](int g) { return (const T*)(sdi + L.off[g]); };
  const int tid = threadIdx.x;
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
  const int n0 = L.nx[L.g0] * L.ny[L.g0];
  bool staged = false;
  for (int col = Bk.bid; col < wp; col += Bk.nb) {
    if (done[col]) continue;
    if (!staged) {
      for (int g = L.g0; g < L.G; ++g) {
        const int n = L.nx[g] * L.ny[g];
        stage_async(sst + 9 * L.off[g], (const T*)L.st[g], 9 * n);
        stage_async(sdi + L.off[g], (const T*)L.dinv[g], n);
      }
      staged = true;
    }
    {
      T* b0 = B(L.g0);
      for (int idx = tid; idx < n0; idx += blockDim.x) cp_async_elem(b0 + idx, bg + idx * wp + col);
    }
    cp_async_wait_all();   // stencils, diagonals and the right-hand side
    __syncthreads();
    T* cur[MAX_LEVELS];
    T* oth[MAX_LEVELS];
    for (int g = L.g0; g < L.G; ++g) {
      const int nx = L.nx[g], ny = L.ny[g], n = nx * ny;
      const bool wm = wmode(g);
      const int lim = wm ? 32 : (int)blockDim.x;
      const bool act = tid < lim;
      const T* st = stg(g);
      const T* dinv = dig(g);
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
      const T* st = stg(g);
      const T* dinv = dig(g);
      const T* b = B(g);
      T* c = cur[g];
      T* o = oth[g];
      const T* xc = cur[g + 1];
      if (act)
        for (int idx = tid; idx < n; idx += lim) {
          const int y = idx / nx, x = idx - y * nx;
          c[idx] += prolong_at(x, y, nxc, nyc, xc);
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
    const T* x0 = cur[L.g0];
    for (int idx = tid; idx < n0; idx += blockDim.x) xg[idx * wp + col] = x0[idx];
    __syncthreads();   // the next column reuses the buffers
  }
}

// r = src (cast; padded columns w..wp-1 zero); acc = ||b||^2 partials. x is
// not cleared: the first update writes it (x = alpha p), and a batch that
// ends before its first iteration scatters zeros.
template <typename TS, typename T>
__device__ __forceinline__ void ph_gather(Blk B, int n, int w, int wp, int k, const TS* __restrict__ src, int lds,
                                          T* __restrict__ r, T (&acc)[VW<T>::N]) {
  constexpr int N = VW<T>::N;
#pragma unroll
  for (int u = 0; u < N; ++u) acc[u] = T(0);
  int cg, node, nstep;
  if (!thread_pos(wp / N, k, B, cg, node, nstep)) return;
  const int c0 = cg * N;
  for (; node < n; node += nstep) {
    Vec<T> v;
#pragma unroll
    for (int u = 0; u < N; ++u) {
      v.a[u] = c0 + u < w ? widen<T>(src[(size_t)node * lds + c0 + u]) : T(0);
      acc[u] += v.a[u] * v.a[u];
    }
    vst(r + node * wp + c0, v);
  }
}

// x (wp columns) -> dst (leading dimension ldd, first w columns); with ctl,
// the PCG iterate: zeros if the batch ended before its first iteration (x
// then was never written)
template <typename T, typename TD>
__device__ __forceinline__ void ph_scatter(Blk B, int n, int w, int wp, int k, const T* __restrict__ x,
                                           TD* __restrict__ dst, int ldd, const InnerCtl* ctl) {
  constexpr int N = VW<T>::N;
  int cg, node, nstep;
  if (!thread_pos(wp / N, k, B, cg, node, nstep)) return;
  const int c0 = cg * N;
  const bool zero = ctl && ctl->it == 0;
  for (; node < n; node += nstep) {
    const Vec<T> v = zero ? vzero<T>() : vld(x + node * wp + c0);
#pragma unroll
    for (int u = 0; u < N; ++u)
      if (c0 + u < w) dst[(size_t)node * ldd + c0 + u] = (TD)v.a[u];
  }
}

// acc = a . b partials per column
template <typename T>
__device__ __forceinline__ void ph_dot(Blk B, int n, int wp, int k, const T* __restrict__ a, const T* __restrict__ b,
                                       const int* __restrict__ done, T (&acc)[VW<T>::N]) {
  constexpr int N = VW<T>::N;
#pragma unroll
  for (int u = 0; u < N; ++u) acc[u] = T(0);
  int cg, node, nstep;
  if (!thread_pos(wp / N, k, B, cg, node, nstep)) return;
  const int c0 = cg * N;
  if (done_mask<N>(done, c0) == (1u << N) - 1) return;
  for (; node < n; node += nstep) {
    const int i = node * wp + c0;
    const Vec<T> av = vld(a + i), bv = vld(b + i);
#pragma unroll
    for (int u = 0; u < N; ++u) acc[u] += av.a[u] * bv.a[u];
  }
}

// p_new = z + beta p_old (p_new = z on the batch's first iteration, p_old not
// read), formed on the fly at the 9 neighbours; q = A_0 p_new; acc = p_new . q
template <typename T>
__device__ __forceinline__ void ph_matvec_p(Blk B, int nx, int ny, int wp, int k, const T* __restrict__ st,
                                            const T* __restrict__ z, const T* __restrict__ pold,
                                            T* __restrict__ pnew, T* __restrict__ q, bool first,
                                            const T* __restrict__ beta, const int* __restrict__ done,
                                            T (&acc)[VW<T>::N]) {
  constexpr int N = VW<T>::N;
#pragma unroll
  for (int u = 0; u < N; ++u) acc[u] = T(0);
  int cg, lx;
  if (!strip_pos(wp / N, k, cg, lx)) return;
  const int c0 = cg * N;
  if (done_mask<N>(done, c0) == (1u << N) - 1) return;
  T bt[N];
#pragma unroll
  for (int u = 0; u < N; ++u) bt[u] = beta[c0 + u];
  const int rs = nx * wp;
  auto pv = [&](int e) {
    Vec<T> v = vld(z + e);
    if (!first) {
      const Vec<T> po = vld(pold + e);
#pragma unroll
      for (int u = 0; u < N; ++u) v.a[u] += bt[u] * po.a[u];
    }
    return v;
  };
  for (StripIter it(B, lx, k, nx, ny); it.valid(); it.next()) {
    if (!it.inside()) continue;
    const int i = it.node * wp + c0;
    const Vec<T> s = stencil9(st + it.node * 9, i, rs, wp, it.node, it.x, it.y, nx, ny,
                              [&](int e, int) { return pv(e); });
    const Vec<T> p = pv(i);
    vst(pnew + i, p);
    vst(q + i, s);
#pragma unroll
    for (int u = 0; u < N; ++u) acc[u] += p.a[u] * s.a[u];
  }
}

// x += alpha p_new; r -= alpha q; acc = r . r. Finished columns keep x and r.
template <typename T>
__device__ __forceinline__ void ph_update_xr(Blk B, int n, int wp, int k, const T* __restrict__ pnew,
                                             const T* __restrict__ q, T* __restrict__ x, T* __restrict__ r,
                                             const T* __restrict__ alpha, const int* __restrict__ done, bool first,
                                             T (&acc)[VW<T>::N]) {
  constexpr int N = VW<T>::N;
#pragma unroll
  for (int u = 0; u < N; ++u) acc[u] = T(0);
  int cg, node, nstep;
  if (!thread_pos(wp / N, k, B, cg, node, nstep)) return;
  const int c0 = cg * N;
  const unsigned dm = done_mask<N>(done, c0);
  if (dm == (1u << N) - 1) {
    if (first)   // columns done at entry: x_0 = 0
      for (; node < n; node += nstep) vst(x + node * wp + c0, vzero<T>());
    return;
  }
  T a[N];
#pragma unroll
  for (int u = 0; u < N; ++u) a[u] = (dm >> u) & 1u ? T(0) : alpha[c0 + u];
  for (; node < n; node += nstep) {
    const int i = node * wp + c0;
    Vec<T> xv = first ? vzero<T>() : vld(x + i);   // the first update writes x (x_0 = 0, not stored)
    Vec<T> rv = vld(r + i);
    const Vec<T> pv = vld(pnew + i), qv = vld(q + i);
#pragma unroll
    for (int u = 0; u < N; ++u) {
      if (!((dm >> u) & 1u)) {
        xv.a[u] += a[u] * pv.a[u];
        rv.a[u] -= a[u] * qv.a[u];
      }
      acc[u] += rv.a[u] * rv.a[u];
    }
    vst(x + i, xv);
    vst(r + i, rv);
  }
}

// The per-column CG scalars the FP32 / FP64 kernels read.
template <typename T>
__device__ __forceinline__ const T* alpha_of(const FinArgs& f) {
  if constexpr (sizeof(T) == 4) return f.alphaf; else return f.alpha;
}
template <typename T>
__device__ __forceinline__ const T* beta_of(const FinArgs& f) {
  if constexpr (sizeof(T) == 4) return f.betaf; else return f.beta;
}

// ------------------------------------------------------- stand-alone kernels ---

template <typename T>
__global__ void __launch_bounds__(1024) k_smooth0(int n, int wp, int k, const T* __restrict__ dinv,
                                                  const T* __restrict__ b, T* __restrict__ x, T om,
                                                  const int* __restrict__ done) {
  ph_smooth0<T>(this_grid(), n, wp, k, dinv, b, x, om, done);
}

template <typename T>
__global__ void __launch_bounds__(1024) k_smooth00(int nx, int ny, int wp, int k, const T* __restrict__ st,
                                                   const T* __restrict__ dinv, const T* __restrict__ b,
                                                   T* __restrict__ x, T om, const int* __restrict__ done) {
  ph_smooth00<T>(this_grid(), nx, ny, wp, k, st, dinv, b, x, om, done);
}

// with DOT also b . xo -> FIN_RHO
template <typename T, bool DOT>
__global__ void __launch_bounds__(1024, DOT ? 1 : 2) k_jacobi(int nx, int ny, int wp, int k, const T* __restrict__ st,
                                                 const T* __restrict__ dinv, const T* __restrict__ b,
                                                 const T* __restrict__ xi, T* __restrict__ xo, T om, FinArgs f) {
  T acc[VW<T>::N];
  ph_jacobi<T, DOT>(this_grid(), nx, ny, wp, k, st, dinv, b, xi, xo, om, f.done, acc);
  if (DOT) reduce_finalize<T, VW<T>::N>(f, acc, wp, k, FIN_RHO);
}

template <typename T>
__global__ void __launch_bounds__(1024) k_resid_restrict_t(int nxf, int nyf, int nxc, int nyc, int wp, int TC,
                                                           const T* __restrict__ st, const T* __restrict__ b,
                                                           const T* __restrict__ x, T* __restrict__ bc,
                                                           const int* __restrict__ done) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ph_resid_restrict<T>(this_grid(), nxf, nyf, nxc, nyc, wp, TC, st, b, x, bc, done, smem_raw);
}

template <typename T, bool DOT>
__global__ void __launch_bounds__(1024) k_prolong_jacobi(int nxf, int nyf, int nxc, int nyc, int wp, int k,
                                                         const T* __restrict__ st, const T* __restrict__ dinv,
                                                         const T* __restrict__ b, const T* __restrict__ x,
                                                         const T* __restrict__ xc, T* __restrict__ xo, T om,
                                                         FinArgs f) {
  T acc[VW<T>::N];
  ph_prolong_jacobi<T, DOT>(this_grid(), nxf, nyf, nxc, nyc, wp, k, st, dinv, b, x, xc, xo, om, f.done, acc);
  if (DOT) reduce_finalize<T, VW<T>::N>(f, acc, wp, k, FIN_RHO);
}

template <typename T>
__global__ void __launch_bounds__(1024) k_vcycle_coarse(CoarseGrids L, int tot, int wp, const T* __restrict__ bg,
                                                        T* __restrict__ xg, T om, int nu,
                                                        const int* __restrict__ done) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ph_coarse<T>(this_grid(), L, tot, wp, bg, xg, om, nu, done, smem_raw);
}

// r = src, ||b||^2 -> FIN_INIT (sets the loop condition; zero columns, the
// padded ones included, are done); x is written by the first update
template <typename TS, typename T>
__global__ void __launch_bounds__(1024) k_gather(int n, int w, int wp, int k, const TS* __restrict__ src, int lds,
                                                 T* __restrict__ r, FinArgs f) {
  T acc[VW<T>::N];
  ph_gather<TS, T>(this_grid(), n, w, wp, k, src, lds, r, acc);
  reduce_finalize<T, VW<T>::N>(f, acc, wp, k, FIN_INIT);
}

// src (leading dimension lds, w columns) -> b (wp columns, padding zero)
template <typename TS, typename T>
__global__ void __launch_bounds__(1024) k_pack(int n, int w, int wp, int k, const TS* __restrict__ src, int lds,
                                               T* __restrict__ b) {
  constexpr int N = VW<T>::N;
  int cg, node, nstep;
  if (!thread_pos(wp / N, k, this_grid(), cg, node, nstep)) return;
  const int c0 = cg * N;
  for (; node < n; node += nstep) {
    Vec<T> v;
#pragma unroll
    for (int u = 0; u < N; ++u) v.a[u] = c0 + u < w ? (T)src[(size_t)node * lds + c0 + u] : T(0);
    vst(b + node * wp + c0, v);
  }
}

template <typename T, typename TD>
__global__ void __launch_bounds__(1024) k_scatter(int n, int w, int wp, int k, const T* __restrict__ x,
                                                  TD* __restrict__ dst, int ldd, const InnerCtl* ctl) {
  ph_scatter<T, TD>(this_grid(), n, w, wp, k, x, dst, ldd, ctl);
}

// a . b per column -> op (used when the finest grid is inside the coarse block)
template <typename T>
__global__ void __launch_bounds__(1024) k_dot_fin(int n, int wp, int k, const T* __restrict__ a, const T* __restrict__ b,
                                                  FinArgs f, int op) {
  T acc[VW<T>::N];
  ph_dot<T>(this_grid(), n, wp, k, a, b, f.done, acc);
  reduce_finalize<T, VW<T>::N>(f, acc, wp, k, op);
}

// p_new (ping-pong by the iteration parity), q = A_0 p_new, p_new . q -> FIN_ALPHA
template <typename T>
__global__ void __launch_bounds__(1024) k_matvec_p(int nx, int ny, int wp, int k, const T* __restrict__ st,
                                                   const T* __restrict__ z, T* __restrict__ pA,
                                                   T* __restrict__ pB, T* __restrict__ q, FinArgs f) {
  const int it = f.ctl->it;
  T acc[VW<T>::N];
  ph_matvec_p<T>(this_grid(), nx, ny, wp, k, st, z, (it & 1) ? pB : pA, (it & 1) ? pA : pB, q, it == 0,
                 beta_of<T>(f), f.done, acc);
  reduce_finalize<T, VW<T>::N>(f, acc, wp, k, FIN_ALPHA);
}

// x += alpha p_new; r -= alpha q; r . r -> FIN_CONV (sets the loop condition)
template <typename T>
__global__ void __launch_bounds__(1024) k_update_xr(int n, int wp, int k, const T* __restrict__ pA,
                                                    const T* __restrict__ pB, const T* __restrict__ q,
                                                    T* __restrict__ x, T* __restrict__ r, FinArgs f) {
  T acc[VW<T>::N];
  const int it = f.ctl->it;
  ph_update_xr<T>(this_grid(), n, wp, k, (it & 1) ? pA : pB, q, x, r, alpha_of<T>(f), f.done, it == 0, acc);
  reduce_finalize<T, VW<T>::N>(f, acc, wp, k, FIN_CONV);
}

__global__ void k_clear_done(int w, int* done) {
  for (int i = threadIdx.x; i < w; i += blockDim.x) done[i] = 0;
}

// ------------------------------------------------ row-pipelined stencils ---
// Large grids, FP32, batches of 64 columns or more: the sweeps as a pipeline of
// row segments staged in shared memory. A block owns strips of PX = 64 nodes
// (plus one halo node on each side) by 64 columns and walks a strip row by
// row. The rows y-1, y, y+1 of the stencil input(s) and the per-row inputs of
// row y sit in a ring of 4 row slots, and the copies of row y+2 (cp.async,
// zero fill outside the grid and the batch) are in flight while row y is
// computed, so the loads do not wait on DRAM latency one node at a time (the
// node-by-node kernels run one 895-thread block per SM at this width, limited
// by registers, and reach 25-40% of HBM). Every value is fetched from global
// memory once per strip; the halo nodes add 2/64. Measured at 511^2 x 716
// columns: the Jacobi sweep with r . z 14% faster than node by node, the
// two-sweep smoother ~25%; the same pipeline for q = A p (two stencil inputs)
// was slower than the node-by-node kernel, and 32-node x 32-column tiles with
// five rows in flight were slower still (128-byte pieces of a node per copy).
namespace pipe {
constexpr int PX = 64;                 // nodes per strip segment
constexpr int PG = 16;                 // float4 column groups per strip (64 columns: 256-byte pieces of a node)
constexpr int RING = 4;                // row slots
constexpr int AHEAD = RING - 3;        // rows in flight beyond y+1
constexpr int NT = PX * PG;            // threads per block
constexpr int HX = PX + 2;             // nodes of a stencil-input row (halo included)
constexpr int SLOT4 = HX * PG;         // float4 per stencil-input slot
constexpr int BSLOT4 = PX * PG;        // float4 per point-input slot
constexpr long long MIN_NODES = 60000; // grids from 255 x 255 up
}  // namespace pipe

enum { PIPE_JACOBI = 0, PIPE_SMOOTH00 = 1 };

// 16- and 4-byte global -> shared copies; a copy marked invalid writes zeros
// and reads nothing (src-size 0; src must still be a mapped address).
__device__ __forceinline__ void cp_async16_z(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async4_z(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most pipe::AHEAD groups (the rows beyond y + 1) are pending
__device__ __forceinline__ void cp_async_wait_ahead() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(pipe::AHEAD) : "memory");
}

template <int OP>
static constexpr size_t pipe_smem_bytes() {
  using namespace pipe;
  return (size_t)RING * SLOT4 * 16 + (OP == PIPE_JACOBI ? (size_t)RING * BSLOT4 * 16 : 0) + (size_t)RING * PX * 9 * 4 +
         (size_t)RING * HX * 4;
}

// OP = PIPE_JACOBI:   xo = x + om D^-1 (b - A x) (X = x, B = b); DOT: b . xo -> FIN_RHO
// OP = PIPE_SMOOTH00: xo = om D^-1 b + om D^-1 (b - om A (D^-1 b)) (X = b), the
//                     first two sweeps from zero
// The block's share of the (strip, row) units is contiguous, strips ordered
// column chunk-major, so every block walks long runs of rows.
template <int OP, bool DOT>
__global__ void __launch_bounds__(pipe::NT, 1)
    k_pipe(int nx, int ny, int wp, const float* __restrict__ st, const float* __restrict__ dinv, const float* X,
           const float* Bv, float* out, float om, FinArgs f) {
  using namespace pipe;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float colacc[1024];
  float4* xr = reinterpret_cast<float4*>(smem_raw);
  float4* br = xr + RING * SLOT4;
  float* sr = reinterpret_cast<float*>(br + (OP == PIPE_JACOBI ? RING * BSLOT4 : 0));
  float* dr = sr + RING * PX * 9;
  const int t = threadIdx.x, grp = t % PG, lx = t / PG;
  const int nseg = (nx + PX - 1) / PX, nch = (wp + 4 * PG - 1) / (4 * PG);
  const long long tot = (long long)nch * nseg * ny;
  long long u = tot * blockIdx.x / gridDim.x;
  const long long u1 = tot * (blockIdx.x + 1) / gridDim.x;
  if (DOT)
    for (int c = t; c < wp; c += NT) colacc[c] = 0.f;
  while (u < u1) {
    const int strip = (int)(u / ny);
    const int ya = (int)(u - (long long)strip * ny);
    const int yb = (int)min((long long)ny, (long long)ya + (u1 - u));
    const int ch = strip / nseg, sg = strip - ch * nseg;
    const int c0 = ch * 4 * PG, x0 = sg * PX;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    auto issue = [&](int r) {
      const int sl = (r + RING) & (RING - 1);
      const bool rowok = r >= 0 && r < ny;
      for (int it = t; it < SLOT4; it += NT) {
        const int j = it / PG, g = it - j * PG;
        const int x = x0 - 1 + j, c = c0 + 4 * g;
        const bool ok = rowok && x >= 0 && x < nx && c < wp;
        const size_t e = ok ? ((size_t)r * nx + x) * wp + c : 0;
        cp_async16_z(&xr[sl * SLOT4 + it], X + e, ok);
      }
      if (OP == PIPE_JACOBI)
        for (int it = t; it < BSLOT4; it += NT) {
          const int j = it / PG, g = it - j * PG;
          const int x = x0 + j, c = c0 + 4 * g;
          const bool ok = rowok && x < nx && c < wp;
          cp_async16_z(&br[sl * BSLOT4 + it], Bv + (ok ? ((size_t)r * nx + x) * wp + c : 0), ok);
        }
      for (int it = t; it < PX * 9; it += NT) {
        const int j = it / 9, x = x0 + j;
        const bool ok = rowok && x < nx;
        cp_async4_z(&sr[sl * PX * 9 + it], st + (ok ? ((size_t)r * nx + x) * 9 + (it - j * 9) : 0), ok);
      }
      for (int it = t; it < HX; it += NT) {
          const int x = x0 - 1 + it;
          const bool ok = rowok && x >= 0 && x < nx;
          cp_async4_z(&dr[sl * HX + it], dinv + (ok ? (size_t)r * nx + x : 0), ok);
        }
    };
    __syncthreads();   // the ring is free (previous strip computed)
    for (int r = ya - 1; r <= ya + AHEAD; ++r) {
      if (r <= yb) issue(r);
      cp_async_commit();
    }
    for (int y = ya; y < yb; ++y) {
      __syncthreads();   // the slot of row y - 2 is read no more
      if (y + AHEAD + 1 <= yb) issue(y + AHEAD + 1);
      cp_async_commit();
      cp_async_wait_ahead();  // this thread's copies of rows <= y + 1
      __syncthreads();        // everyone's
      const int x = x0 + lx, c = c0 + 4 * grp;
      if (x < nx && c < wp) {
        const int s1 = y & (RING - 1);
        const float* s9 = sr + s1 * PX * 9 + lx * 9;
        auto val = [&](int sl, int j) -> float4 {   // stencil input at slot sl, strip node j (0 .. HX-1)
          const float4 v = xr[sl * SLOT4 + j * PG + grp];
          if (OP == PIPE_SMOOTH00) {
            const float d = dr[sl * HX + j];
            return make_float4(v.x * d, v.y * d, v.z * d, v.w * d);
          }
          return v;
        };
        float4 ax = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
          const int sl = (y + dy + RING) & (RING - 1);
#pragma unroll
          for (int dx = -1; dx <= 1; ++dx) {
            const float a = s9[(dy + 1) * 3 + (dx + 1)];
            const float4 v = val(sl, lx + 1 + dx);
            ax.x = fmaf(a, v.x, ax.x);
            ax.y = fmaf(a, v.y, ax.y);
            ax.z = fmaf(a, v.z, ax.z);
            ax.w = fmaf(a, v.w, ax.w);
          }
        }
        const size_t e = ((size_t)y * nx + x) * wp + c;
        if (OP == PIPE_JACOBI) {
          const float4 xv = xr[s1 * SLOT4 + (lx + 1) * PG + grp];
          const float4 bv = br[s1 * BSLOT4 + lx * PG + grp];
          const float dd = om * dr[s1 * HX + lx + 1];
          const float4 o = make_float4(xv.x + dd * (bv.x - ax.x), xv.y + dd * (bv.y - ax.y), xv.z + dd * (bv.z - ax.z),
                                       xv.w + dd * (bv.w - ax.w));
          *reinterpret_cast<float4*>(out + e) = o;
          if (DOT) {
            acc[0] += bv.x * o.x;
            acc[1] += bv.y * o.y;
            acc[2] += bv.z * o.z;
            acc[3] += bv.w * o.w;
          }
        } else {
          const float4 bv = xr[s1 * SLOT4 + (lx + 1) * PG + grp];
          const float di = om * dr[s1 * HX + lx + 1];
          *reinterpret_cast<float4*>(out + e) =
              make_float4(di * bv.x + di * (bv.x - om * ax.x), di * bv.y + di * (bv.y - om * ax.y),
                          di * bv.z + di * (bv.z - om * ax.z), di * bv.w + di * (bv.w - om * ax.w));
        }
      }
    }
    if (DOT) {
      // the strip's partial sums per column (fixed order: nodes of the strip
      // in lx order) into colacc; the ring holds nothing needed any more (no
      // copy is pending: the last AHEAD groups of the strip were empty)
      __syncthreads();
      float* red = reinterpret_cast<float*>(xr);   // [PX][4 PG]
#pragma unroll
      for (int q = 0; q < 4; ++q) red[lx * 4 * PG + 4 * grp + q] = acc[q];
      __syncthreads();
      if (t < 4 * PG && c0 + t < wp) {
        float sum = 0.f;
        for (int j = 0; j < PX; ++j) sum += red[j * 4 * PG + t];
        colacc[c0 + t] += sum;
      }
    }
    u += yb - ya;
  }
  if (DOT) {
    __syncthreads();
    float* part = (float*)f.part;
    for (int c = t; c < wp; c += NT) part[(size_t)blockIdx.x * f.ldp + c] = colacc[c];
    __threadfence();
    if (last_block(&f.ctl->ticket)) fin_columns<float>(f, FIN_RHO, wp, gridDim.x);
  }
}

// The residual and its restriction in the same row pipeline: bc = P^T (b - A x)
// on the coarse grid of every other row. A block owns strips of 32 coarse nodes
// (fine nodes x0 .. x0 + 64 of their restriction stencils, x0 = 64 * strip) by
// 64 columns and a contiguous run of coarse rows [Ya, Yb); it walks the fine
// rows 2 Ya .. 2 Yb, forms each residual row once into a ring of 3 rows, and
// after fine row 2Y + 2 writes coarse row Y from rows 2Y, 2Y + 1, 2Y + 2.
// Inputs per fine row: x on nodes x0 - 1 .. x0 + 65 (ring of 4, the row after
// next in flight), b and the stencils on x0 .. x0 + 64.
namespace rpipe {
constexpr int RX = pipe::PX + 1;       // residual nodes of a strip: x0 .. x0 + 64
constexpr int XX = RX + 2;             // x nodes: x0 - 1 .. x0 + 65
constexpr int CX = pipe::PX / 2;       // coarse nodes per strip
constexpr int PG = pipe::PG, RING = 4, NT = pipe::NT;
constexpr int XSLOT = XX * PG, BSLOT = RX * PG, RSLOT = RX * PG;
}  // namespace rpipe

static constexpr size_t rpipe_smem_bytes() {
  using namespace rpipe;
  return (size_t)RING * XSLOT * 16 + (size_t)RING * BSLOT * 16 + (size_t)3 * RSLOT * 16 + (size_t)RING * RX * 9 * 4;
}

__global__ void __launch_bounds__(rpipe::NT, 1)
    k_pipe_restrict(int nxf, int nyf, int nxc, int nyc, int wp, const float* __restrict__ st, const float* X,
                    const float* Bv, float* bc) {
  using namespace rpipe;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* xr = reinterpret_cast<float4*>(smem_raw);   // [RING][XX][PG]
  float4* br = xr + RING * XSLOT;                      // [RING][RX][PG]
  float4* rr = br + RING * BSLOT;                      // [3][RX][PG] residual rows
  float* sr = reinterpret_cast<float*>(rr + 3 * RSLOT);   // [RING][RX * 9]
  const int t = threadIdx.x;
  const int nseg = (nxc + CX - 1) / CX, nch = (wp + 4 * PG - 1) / (4 * PG);
  const long long tot = (long long)nch * nseg * nyc;
  long long u = tot * blockIdx.x / gridDim.x;
  const long long u1 = tot * (blockIdx.x + 1) / gridDim.x;
  while (u < u1) {
    const int strip = (int)(u / nyc);
    const int Ya = (int)(u - (long long)strip * nyc);
    const int Yb = (int)min((long long)nyc, (long long)Ya + (u1 - u));
    const int ch = strip / nseg, sg = strip - ch * nseg;
    const int c0 = ch * 4 * PG, x0 = sg * pipe::PX;
    const int ya = 2 * Ya, yb = 2 * Yb;   // fine rows whose residuals are formed: ya .. yb
    auto issue = [&](int r) {
      const int sl = r & (RING - 1);
      const bool rowok = r >= 0 && r < nyf;
      for (int it = t; it < XSLOT; it += NT) {
        const int j = it / PG, g = it - j * PG;
        const int x = x0 - 1 + j, c = c0 + 4 * g;
        const bool ok = rowok && x >= 0 && x < nxf && c < wp;
        cp_async16_z(&xr[sl * XSLOT + it], X + (ok ? ((size_t)r * nxf + x) * wp + c : 0), ok);
      }
      for (int it = t; it < BSLOT; it += NT) {
        const int j = it / PG, g = it - j * PG;
        const int x = x0 + j, c = c0 + 4 * g;
        const bool ok = rowok && x < nxf && c < wp;
        cp_async16_z(&br[sl * BSLOT + it], Bv + (ok ? ((size_t)r * nxf + x) * wp + c : 0), ok);
      }
      for (int it = t; it < RX * 9; it += NT) {
        const int j = it / 9, x = x0 + j;
        const bool ok = rowok && x < nxf;
        cp_async4_z(&sr[sl * RX * 9 + it], st + (ok ? ((size_t)r * nxf + x) * 9 + (it - j * 9) : 0), ok);
      }
    };
    __syncthreads();   // the rings are free (previous strip done)
    for (int r = ya - 1; r <= ya + 1; ++r) {
      if (r <= yb + 1) issue(r);
      cp_async_commit();
    }
    for (int y = ya; y <= yb; ++y) {
      __syncthreads();   // the slot of row y - 2 is read no more
      if (y + 2 <= yb + 1) issue(y + 2);
      cp_async_commit();
      cp_async_wait_ahead();
      __syncthreads();
      // residual row y (zero outside the fine grid)
      const int s1 = y & (RING - 1), s0 = (y + RING - 1) & (RING - 1), s2 = (y + 1) & (RING - 1);
      const int rs = y % 3;
      for (int it = t; it < RSLOT; it += NT) {
        const int j = it / PG, g = it - j * PG;
        const int x = x0 + j;
        float4 res = make_float4(0.f, 0.f, 0.f, 0.f);
        if (y < nyf && x < nxf && c0 + 4 * g < wp) {
          const float* s9 = sr + s1 * RX * 9 + j * 9;
          float4 ax = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int dy = 0; dy < 3; ++dy) {
            const int sl = dy == 0 ? s0 : (dy == 1 ? s1 : s2);
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
              const float a = s9[dy * 3 + dx];
              const float4 v = xr[sl * XSLOT + (j + dx) * PG + g];
              ax.x = fmaf(a, v.x, ax.x);
              ax.y = fmaf(a, v.y, ax.y);
              ax.z = fmaf(a, v.z, ax.z);
              ax.w = fmaf(a, v.w, ax.w);
            }
          }
          const float4 bv = br[s1 * BSLOT + j * PG + g];
          res = make_float4(bv.x - ax.x, bv.y - ax.y, bv.z - ax.z, bv.w - ax.w);
        }
        rr[rs * RSLOT + it] = res;
      }
      // coarse row Y = y / 2 - 1 once fine rows 2Y .. 2Y + 2 are formed
      if (!(y & 1) && y >= ya + 2) {
        __syncthreads();
        const int Y = y / 2 - 1;
        const int ra = (y - 2) % 3, rb = (y - 1) % 3, rc = rs;
        for (int it = t; it < CX * PG; it += NT) {
          const int Xl = it / PG, g = it - Xl * PG;
          const int Xc = x0 / 2 + Xl, c = c0 + 4 * g;
          if (Xc >= nxc || c >= wp) continue;
          const int jc = 2 * Xl + 1;   // fine node 2X + 1 within the strip
          float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int dy = 0; dy < 3; ++dy) {
            const int rsl = dy == 0 ? ra : (dy == 1 ? rb : rc);
            const float wy = dy == 1 ? 1.f : 0.5f;
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
              const float wgt = wy * (dx == 0 ? 1.f : 0.5f);
              const float4 v = rr[rsl * RSLOT + (jc + dx) * PG + g];
              acc.x = fmaf(wgt, v.x, acc.x);
              acc.y = fmaf(wgt, v.y, acc.y);
              acc.z = fmaf(wgt, v.z, acc.z);
              acc.w = fmaf(wgt, v.w, acc.w);
            }
          }
          *reinterpret_cast<float4*>(bc + ((size_t)Y * nxc + Xc) * wp + c) = acc;
        }
      }
    }
    u += Yb - Ya;
  }
}

// The coarse correction with the first post-smoothing sweep in the row
// pipeline: x' = x + P xc, xo = x' + om D^-1 (b - A x') (no dot). Besides the
// fine rows (x with halo, b, stencils, diagonals: rings of 4 as in k_pipe) a
// ring of 4 coarse rows holds xc on the coarse nodes x0/2 - 2 .. x0/2 + 32 that
// the strip's interpolation patches touch; coarse rows advance one per two fine
// rows, each fetched two fine steps before its first use. The correction is
// formed as in the node-by-node kernel: per fine node the 3 x 3 coarse patch
// and the weights K = Wy^T S Wx.
namespace ppipe {
constexpr int CN = pipe::PX / 2 + 3;   // coarse nodes of a strip's patches
constexpr int CSLOT = CN * pipe::PG;
}  // namespace ppipe

static constexpr size_t ppipe_smem_bytes() {
  return pipe_smem_bytes<PIPE_JACOBI>() + (size_t)pipe::RING * ppipe::CSLOT * 16;
}

// interpolation weight of patch entry a (0..2) for the fine point at offset d
// (-1..1) from a fine coordinate of parity odd (coarse node X on fine 2X + 1)
__device__ __forceinline__ float pp_w(bool odd, int d, int a) {
  if (odd) return d < 0 ? (a < 2 ? 0.5f : 0.f) : d == 0 ? (a == 1 ? 1.f : 0.f) : (a > 0 ? 0.5f : 0.f);
  return d < 0 ? (a == 1 ? 1.f : 0.f) : d == 0 ? (a > 0 ? 0.5f : 0.f) : (a == 2 ? 1.f : 0.f);
}

__global__ void __launch_bounds__(pipe::NT, 1)
    k_pipe_prolong(int nx, int ny, int nxc, int nyc, int wp, const float* __restrict__ st,
                   const float* __restrict__ dinv, const float* X, const float* Bv, const float* XC, float* out,
                   float om) {
  using namespace pipe;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* xr = reinterpret_cast<float4*>(smem_raw);
  float4* br = xr + RING * SLOT4;
  float* sr = reinterpret_cast<float*>(br + RING * BSLOT4);
  float* dr = sr + RING * PX * 9;
  float4* cr = reinterpret_cast<float4*>(dr + RING * HX);   // [RING][CN][PG] coarse rows
  const int t = threadIdx.x, grp = t % PG, lx = t / PG;
  const int nseg = (nx + PX - 1) / PX, nch = (wp + 4 * PG - 1) / (4 * PG);
  const long long tot = (long long)nch * nseg * ny;
  long long u = tot * blockIdx.x / gridDim.x;
  const long long u1 = tot * (blockIdx.x + 1) / gridDim.x;
  while (u < u1) {
    const int strip = (int)(u / ny);
    const int ya = (int)(u - (long long)strip * ny);
    const int yb = (int)min((long long)ny, (long long)ya + (u1 - u));
    const int ch = strip / nseg, sg = strip - ch * nseg;
    const int c0 = ch * 4 * PG, x0 = sg * PX, X0 = x0 / 2 - 2;   // first coarse node of the patches
    auto issue = [&](int r) {   // fine row r
      const int sl = r & (RING - 1);
      const bool rowok = r >= 0 && r < ny;
      for (int it = t; it < SLOT4; it += NT) {
        const int j = it / PG, g = it - j * PG;
        const int x = x0 - 1 + j, c = c0 + 4 * g;
        const bool ok = rowok && x >= 0 && x < nx && c < wp;
        cp_async16_z(&xr[sl * SLOT4 + it], X + (ok ? ((size_t)r * nx + x) * wp + c : 0), ok);
      }
      for (int it = t; it < BSLOT4; it += NT) {
        const int j = it / PG, g = it - j * PG;
        const int x = x0 + j, c = c0 + 4 * g;
        const bool ok = rowok && x < nx && c < wp;
        cp_async16_z(&br[sl * BSLOT4 + it], Bv + (ok ? ((size_t)r * nx + x) * wp + c : 0), ok);
      }
      for (int it = t; it < PX * 9; it += NT) {
        const int j = it / 9, x = x0 + j;
        const bool ok = rowok && x < nx;
        cp_async4_z(&sr[sl * PX * 9 + it], st + (ok ? ((size_t)r * nx + x) * 9 + (it - j * 9) : 0), ok);
      }
      for (int it = t; it < HX; it += NT) {
        const int x = x0 - 1 + it;
        const bool ok = rowok && x >= 0 && x < nx;
        cp_async4_z(&dr[sl * HX + it], dinv + (ok ? (size_t)r * nx + x : 0), ok);
      }
    };
    auto issue_c = [&](int R) {   // coarse row R
      const int sl = R & (RING - 1);
      const bool rowok = R >= 0 && R < nyc;
      for (int it = t; it < ppipe::CSLOT; it += NT) {
        const int j = it / PG, g = it - j * PG;
        const int Xc = X0 + j, c = c0 + 4 * g;
        const bool ok = rowok && Xc >= 0 && Xc < nxc && c < wp;
        cp_async16_z(&cr[sl * ppipe::CSLOT + it], XC + (ok ? ((size_t)R * nxc + Xc) * wp + c : 0), ok);
      }
    };
    // coarse rows needed by fine row y: ((y-1)>>1) - 1 .. ((y-1)>>1) + 1
    int cnext = ((ya - 1) >> 1) - 1;
    const int clast = ((yb - 2) >> 1) + 1;
    __syncthreads();
    for (int r = ya - 1; r <= ya + 1; ++r) {
      if (r <= yb) issue(r);
      const int need = ((r + 1 - 1) >> 1) + 1;   // coarse rows needed by fine row r + 1
      while (cnext <= need && cnext <= clast) issue_c(cnext++);
      cp_async_commit();
    }
    for (int y = ya; y < yb; ++y) {
      __syncthreads();
      if (y + 2 <= yb) issue(y + 2);
      {
        const int need = ((y + 3 - 1) >> 1) + 1;   // coarse rows needed by fine row y + 3
        while (cnext <= need && cnext <= clast) issue_c(cnext++);
      }
      cp_async_commit();
      cp_async_wait_ahead();
      __syncthreads();
      const int x = x0 + lx, c = c0 + 4 * grp;
      if (x < nx && c < wp) {
        const int s1 = y & (RING - 1);
        const float* s9 = sr + s1 * PX * 9 + lx * 9;
        float4 ax = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
          const int sl = (y + dy + RING) & (RING - 1);
#pragma unroll
          for (int dx = -1; dx <= 1; ++dx) {
            const float a = s9[(dy + 1) * 3 + (dx + 1)];
            const float4 v = xr[sl * SLOT4 + (lx + 1 + dx) * PG + grp];
            ax.x = fmaf(a, v.x, ax.x);
            ax.y = fmaf(a, v.y, ax.y);
            ax.z = fmaf(a, v.z, ax.z);
            ax.w = fmaf(a, v.w, ax.w);
          }
        }
        // coarse correction: patch rows Yb - 1 + a, columns Xb - 1 + c
        const bool oy = y & 1, ox = x & 1;
        const int Yb = (y - 1) >> 1, Xb = (x - 1) >> 1;
        float t1[3][3];   // t1[dy][cc] = sum_dx s[dy][dx] wx(dx, cc), s masked to the grid
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
          const bool iny = y + dy - 1 >= 0 && y + dy - 1 < ny;
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) {
            float acc = 0.f;
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
              const bool inx = x + dx - 1 >= 0 && x + dx - 1 < nx;
              acc += (iny && inx ? s9[dy * 3 + dx] : 0.f) * pp_w(ox, dx - 1, cc);
            }
            t1[dy][cc] = acc;
          }
        }
        float4 apc = make_float4(0.f, 0.f, 0.f, 0.f), pc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int aa = 0; aa < 3; ++aa) {
          const int ar = (oy || aa > 0) ? aa : 1;   // all-zero weights: a valid slot instead
          const int sl = (Yb - 1 + ar + RING) & (RING - 1);
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) {
            const int ccr = (ox || cc > 0) ? cc : 1;
            const float K = pp_w(oy, -1, aa) * t1[0][cc] + pp_w(oy, 0, aa) * t1[1][cc] + pp_w(oy, 1, aa) * t1[2][cc];
            const float w0 = pp_w(oy, 0, aa) * pp_w(ox, 0, cc);
            const float4 v = cr[sl * ppipe::CSLOT + (Xb - 1 + ccr - X0) * PG + grp];
            apc.x = fmaf(K, v.x, apc.x);
            apc.y = fmaf(K, v.y, apc.y);
            apc.z = fmaf(K, v.z, apc.z);
            apc.w = fmaf(K, v.w, apc.w);
            pc.x = fmaf(w0, v.x, pc.x);
            pc.y = fmaf(w0, v.y, pc.y);
            pc.z = fmaf(w0, v.z, pc.z);
            pc.w = fmaf(w0, v.w, pc.w);
          }
        }
        const float4 xv0 = xr[s1 * SLOT4 + (lx + 1) * PG + grp];
        const float4 xv = make_float4(xv0.x + pc.x, xv0.y + pc.y, xv0.z + pc.z, xv0.w + pc.w);
        const float4 bv = br[s1 * BSLOT4 + lx * PG + grp];
        const float dd = om * dr[s1 * HX + lx + 1];
        *reinterpret_cast<float4*>(out + ((size_t)y * nx + x) * wp + c) =
            make_float4(xv.x + dd * (bv.x - (ax.x + apc.x)), xv.y + dd * (bv.y - (ax.y + apc.y)),
                        xv.z + dd * (bv.z - (ax.z + apc.z)), xv.w + dd * (bv.w - (ax.w + apc.w)));
      }
    }
    u += yb - ya;
  }
}

// ------------------------------------------------------------ host side ---

// Row-pipelined sweeps (k_pipe: the Jacobi sweeps and the two sweeps from
// zero) on grids of at least pipe::MIN_NODES nodes, FP32 batches of 64 columns
// or more; smaller grids and narrower batches keep the node-by-node kernels.
template <typename T>
static bool use_pipe(const sg_problem* h, const GridLevel& G, int wp) {
  return sizeof(T) == 4 && !h->pipe_off && (long long)G.n >= pipe::MIN_NODES && wp >= 4 * pipe::PG;
}

template <int OP, bool DOT>
static int launch_pipe(sg_problem* h, const GridLevel& G, int wp, const float* st, const float* dinv, const float* X,
                       const float* Bv, float* out, float om, const FinArgs& f, cudaStream_t s) {
  auto kern = k_pipe<OP, DOT>;
  const size_t smem = pipe_smem_bytes<OP>();
  SG_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  SG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, pipe::NT, smem));
  const int grid = h->num_sms * std::max(per_sm, 1);
  { kern<<<grid, pipe::NT, smem, s>>>(G.nx, G.ny, wp, st, dinv, X, Bv, out, om, f); ::sghsc::note_launch(); }
  SG_CHECK_LAUNCH();
  return SG_OK;
}

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
  wcap = (wcap + 3) / 4 * 4;   // room for the padded width of either precision
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
  iw.wcap = wcap;   // only once every buffer exists: a failed allocation leaves no capacity
  return SG_OK;
}

int check_prec_opts(const sg_prec_opts& o) {
  if (o.nu < 1 || o.nu > 16 || !(o.omega > 0.0) || o.inner_maxit < 1 || o.inner_fixed_iters < 0 ||
      !(o.inner_tol >= 0.0) || (o.m0 != SG_M0_VCYCLE && o.m0 != SG_M0_DIAG) || !(o.level_tol >= 0.0) ||
      o.level_maxit < 1 || o.level_maxit > 100000 || (o.df64 != 0 && o.df64 != 1) || o.md_m0 < 0 || o.md_m0 > 3) {
    set_error("prec opts: need 1 <= nu <= 16, omega > 0, inner_maxit >= 1, inner_tol >= 0, m0 0 or 1, "
              "level_tol >= 0, 1 <= level_maxit <= 100000, df64 0 or 1, md_m0 0..3");
    return SG_ERR_INVALID_ARG;
  }
  return SG_OK;
}

int check_inner_support(const sg_problem* h, const sg_prec_opts& o, const char* name) {
  if (h->grids.empty()) {
    set_error("%s: the inner solves need the Q1 grid of A_0 (a mesh given to sg_setup with the 9-point pattern)",
              name);
    return SG_ERR_UNSUPPORTED;
  }
  if (o.m0 == SG_M0_VCYCLE && !h->mg_full) {
    set_error("%s: the multigrid M_0 needs a power-of-two square mesh (use m0 = SG_M0_DIAG)", name);
    return SG_ERR_UNSUPPORTED;
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
  f.count_iacc = 1;
  return f;
}

template <typename T>
static int launch_coarse(sg_problem* h, int g0, const T* b, T* x, int wp, const sg_prec_opts& o, const int* done,
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
  const size_t smem = coarse_smem_bytes<T>(tot);
  SG_TRY_CUDA(cudaFuncSetAttribute(k_vcycle_coarse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  { k_vcycle_coarse<T><<<wp, 1024, smem, s>>>(L, tot, wp, b, x, (T)o.omega, o.nu, done); ::sghsc::note_launch(); }
  SG_CHECK_LAUNCH();
  return SG_OK;
}

// Tile edge of the tiled restriction from grid G to grid C: the largest
// (<= 16) whose fine footprint (2TC+1)^2 times the column groups stays within
// 2048 residuals per block, shrunk while that leaves fewer tiles than SMs.
static int restrict_tile(const sg_problem* h, const GridLevel& C, int ng) {
  auto items = [&](int tc) { return (2 * tc + 1) * (2 * tc + 1) * ng; };
  auto tiles = [&](int tc) { return ceil_div(C.nx, tc) * ceil_div(C.ny, tc); };
  int tc = 16;
  while (tc > 1 && items(tc) > 2048) --tc;
  while (tc > 1 && tiles(tc) < h->num_sms) --tc;
  return tc;
}

// Tiled residual + restriction (k_resid_restrict_t).
template <typename T>
static int launch_resid_restrict(sg_problem* h, const GridLevel& G, const GridLevel& C, int wp, const T* st,
                                 const T* b, const T* x, T* bc, const int* done, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (use_pipe<T>(h, G, wp)) {
      const size_t smem = rpipe_smem_bytes();
      SG_TRY_CUDA(cudaFuncSetAttribute(k_pipe_restrict, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      { k_pipe_restrict<<<h->num_sms, rpipe::NT, smem, s>>>(G.nx, G.ny, C.nx, C.ny, wp, st, x, b, bc); ::sghsc::note_launch(); }
      SG_CHECK_LAUNCH();
      return SG_OK;
    }
  }
  const int ng = wp / VW<T>::N;
  const int tc = restrict_tile(h, C, ng);
  const int items = (2 * tc + 1) * (2 * tc + 1) * ng;
  const int bdim = std::min(1024, (items + 31) / 32 * 32);
  const size_t smem = (size_t)items * 16;
  auto tiles = [&](int t) { return ceil_div(C.nx, t) * ceil_div(C.ny, t); };
  SG_TRY_CUDA(cudaFuncSetAttribute(k_resid_restrict_t<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  SG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_resid_restrict_t<T>, bdim, smem));
  const int grid = std::max(1, std::min(tiles(tc), h->num_sms * std::max(per_sm, 1)));
  { k_resid_restrict_t<T><<<grid, bdim, smem, s>>>(G.nx, G.ny, C.nx, C.ny, wp, tc, st, b, x, bc, done); ::sghsc::note_launch(); }
  SG_CHECK_LAUNCH();
  return SG_OK;
}

// One weighted-Jacobi sweep xo = xi + om D^-1 (b - A xi) on grid G (with DOT
// also b . xo into f's reduction): row-pipelined where use_pipe allows.
template <typename T, bool DOT>
static int jacobi_sweep(sg_problem* h, InnerWork& iw, const GridLevel& G, const Shape& sh, int wp, const T* st,
                        const T* dinv, const T* b, const T* xi, T* xo, T om, const FinArgs& f, cudaStream_t s) {
  (void)iw;
  if constexpr (sizeof(T) == 4) {
    if (use_pipe<T>(h, G, wp))
      return launch_pipe<PIPE_JACOBI, DOT>(h, G, wp, st, dinv, xi, b, xo, om, f, s);
  }
  if (DOT) {
    { k_jacobi<T, true><<<sh.grid, sh.bdim, 0, s>>>(G.nx, G.ny, wp, sh.k, st, dinv, b, xi, xo, om, f); ::sghsc::note_launch(); }
  } else {
    { const Shape f_ = fit(h, sh, k_jacobi<T, false>); k_jacobi<T, false><<<f_.grid, f_.bdim, 0, s>>>(G.nx, G.ny, wp, f_.k, st, dinv, b, xi, xo, om, f); ::sghsc::note_launch(); }
  }
  SG_CHECK_LAUNCH();
  return SG_OK;
}

// One V-cycle on grid g applied to b (zero initial guess), all blocks with the
// padded width wp. *out receives the buffer holding the result (x or xt). With
// fdot (finest grid only) the last kernel also reduces b . result into FIN_RHO.
template <typename T>
static int vcycle(sg_problem* h, InnerWork& iw, int g, const T* b, T* x, T* xt, int wp, const sg_prec_opts& o,
                  cudaStream_t s, const FinArgs* fdot, const T** out) {
  constexpr int N = VW<T>::N;
  const int ng = wp / N;
  const T om = (T)o.omega;
  FinArgs fz = make_fin(h, iw, o);
  if (o.m0 == SG_M0_DIAG) {
    // the diagonal mean-value preconditioner (Sec. 6 tried none, diagonal and
    // LU): x = D^{-1} b, the first Jacobi sweep from zero with unit damping
    const GridLevel& G = h->grids[g];
    const T* dinv = sizeof(T) == 8 ? (const T*)G.dinv64 : (const T*)G.dinv32;
    const Shape sh = make_shape(h, G.n, ng);
    { const Shape f_ = fit(h, sh, k_smooth0<T>); k_smooth0<T><<<f_.grid, f_.bdim, 0, s>>>(G.n, wp, f_.k, dinv, b, x, T(1), iw.done); ::sghsc::note_launch(); }
    if (fdot) {
      const Shape shd = make_shape(h, G.n, ng, 1);
      { k_dot_fin<T><<<shd.grid, shd.bdim, 0, s>>>(G.n, wp, shd.k, b, x, *fdot, FIN_RHO); ::sghsc::note_launch(); }
    }
    SG_CHECK_LAUNCH();
    *out = x;
    return SG_OK;
  }
  if (g >= h->cb_level) {
    SG_TRY(launch_coarse<T>(h, g, b, x, wp, o, iw.done, s));
    if (fdot) {
      const Shape sh = make_shape(h, h->grids[g].n, ng, 1);
      { k_dot_fin<T><<<sh.grid, sh.bdim, 0, s>>>(h->grids[g].n, wp, sh.k, b, x, *fdot, FIN_RHO); ::sghsc::note_launch(); }
    }
    *out = x;
    return SG_OK;
  }
  const GridLevel& G = h->grids[g];
  const GridLevel& C = h->grids[g + 1];
  const T* st = sizeof(T) == 8 ? (const T*)G.st64 : (const T*)G.st32;
  const T* dinv = sizeof(T) == 8 ? (const T*)G.dinv64 : (const T*)G.dinv32;
  const Shape sh = make_shape(h, G.n, ng);
  const Shape shd = make_shape(h, G.n, ng, 1);   // kernels that end in a reduction
  T* cur = x;
  T* oth = xt;
  if (o.nu == 1) {
    { const Shape f_ = fit(h, sh, k_smooth0<T>); k_smooth0<T><<<f_.grid, f_.bdim, 0, s>>>(G.n, wp, f_.k, dinv, b, cur, om, iw.done); ::sghsc::note_launch(); }
  } else {
    if constexpr (sizeof(T) == 4) {
      if (use_pipe<T>(h, G, wp))
        SG_TRY((launch_pipe<PIPE_SMOOTH00, false>(h, G, wp, st, dinv, b, nullptr, cur, om, fz, s)));
      else
        { const Shape f_ = fit(h, sh, k_smooth00<T>); k_smooth00<T><<<f_.grid, f_.bdim, 0, s>>>(G.nx, G.ny, wp, f_.k, st, dinv, b, cur, om, iw.done); ::sghsc::note_launch(); }
    } else {
      { const Shape f_ = fit(h, sh, k_smooth00<T>); k_smooth00<T><<<f_.grid, f_.bdim, 0, s>>>(G.nx, G.ny, wp, f_.k, st, dinv, b, cur, om, iw.done); ::sghsc::note_launch(); }
    }
    for (int it = 2; it < o.nu; ++it) {
      SG_TRY((jacobi_sweep<T, false>(h, iw, G, sh, wp, st, dinv, b, cur, oth, om, fz, s)));
      std::swap(cur, oth);
    }
  }
  T* cb = (T*)iw.cb[g + 1];
  SG_TRY(launch_resid_restrict<T>(h, G, C, wp, st, b, cur, cb, iw.done, s));
  const T* xc = nullptr;
  SG_TRY(vcycle<T>(h, iw, g + 1, cb, (T*)iw.cx[g + 1], (T*)iw.cxt[g + 1], wp, o, s, nullptr, &xc));
  bool piped = false;
  if constexpr (sizeof(T) == 4) {
    if (use_pipe<T>(h, G, wp) && !(o.nu == 1 && fdot)) {
      const size_t smem = ppipe_smem_bytes();
      SG_TRY_CUDA(cudaFuncSetAttribute(k_pipe_prolong, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      { k_pipe_prolong<<<h->num_sms, pipe::NT, smem, s>>>(G.nx, G.ny, C.nx, C.ny, wp, st, dinv, cur, b, xc, oth, om); ::sghsc::note_launch(); }
      SG_CHECK_LAUNCH();
      piped = true;
    }
  }
  if (piped) {
  } else if (o.nu == 1 && fdot) {
    { k_prolong_jacobi<T, true><<<shd.grid, shd.bdim, 0, s>>>(G.nx, G.ny, C.nx, C.ny, wp, shd.k, st, dinv, b, cur, xc, oth, om, *fdot); ::sghsc::note_launch(); }
  } else {
    { const Shape f_ = fit(h, sh, k_prolong_jacobi<T, false>); k_prolong_jacobi<T, false><<<f_.grid, f_.bdim, 0, s>>>(G.nx, G.ny, C.nx, C.ny, wp, f_.k, st, dinv, b, cur, xc, oth, om, fz); ::sghsc::note_launch(); }
  }
  std::swap(cur, oth);
  for (int it = 1; it < o.nu; ++it) {
    if (it == o.nu - 1 && fdot)
      SG_TRY((jacobi_sweep<T, true>(h, iw, G, shd, wp, st, dinv, b, cur, oth, om, *fdot, s)));
    else
      SG_TRY((jacobi_sweep<T, false>(h, iw, G, sh, wp, st, dinv, b, cur, oth, om, fz, s)));
    std::swap(cur, oth);
  }
  SG_CHECK_LAUNCH();
  *out = cur;
  return SG_OK;
}

template <typename T>
static int inner_solve_t(sg_problem* h, const void* src, int ld_src, int src_t, void* dst, int ld_dst, int dst_t,
                         int w, const sg_prec_opts& o, cudaStream_t s) {
  constexpr int N = VW<T>::N;
  InnerWork& iw = sizeof(T) == 8 ? h->iw64 : h->iw32;
  const GridLevel& G = h->grids[0];
  const int wp = padded_width<T>(w), ng = wp / N;
  const Shape sh = make_shape(h, G.n, ng, 1);    // gather / matvec / update end in reductions
  const Shape shs = make_shape(h, G.n, ng);
  T* x = (T*)iw.x;
  T* r = (T*)iw.r;
  T* q = (T*)iw.q;
  T* pA = (T*)iw.pA;
  T* pB = (T*)iw.pB;
  const T* st = sizeof(T) == 8 ? (const T*)G.st64 : (const T*)G.st32;
  FinArgs fa = make_fin(h, iw, o);
  auto pre = [&](cudaStream_t ps, const LoopCtl& lc) -> int {
    FinArgs f = fa;
    f.cond = lc.cond;
    f.has_cond = lc.has_cond;
    f.flag = lc.flag;
    if (src_t == SG_F64)
      { k_gather<double, T><<<sh.grid, sh.bdim, 0, ps>>>(G.n, w, wp, sh.k, (const double*)src, ld_src, r, f); ::sghsc::note_launch(); }
    else
      { k_gather<float, T><<<sh.grid, sh.bdim, 0, ps>>>(G.n, w, wp, sh.k, (const float*)src, ld_src, r, f); ::sghsc::note_launch(); }
    SG_CHECK_LAUNCH();
    return SG_OK;
  };
  auto body = [&](cudaStream_t bs, const LoopCtl& lc) -> int {
    FinArgs f = fa;
    f.cond = lc.cond;
    f.has_cond = lc.has_cond;
    f.flag = lc.flag;
    const T* z = nullptr;
    SG_TRY(vcycle<T>(h, iw, 0, r, (T*)iw.z, (T*)iw.zt, wp, o, bs, &f, &z));
    { k_matvec_p<T><<<sh.grid, sh.bdim, 0, bs>>>(G.nx, G.ny, wp, sh.k, st, z, pA, pB, q, f); ::sghsc::note_launch(); }
    { k_update_xr<T><<<sh.grid, sh.bdim, 0, bs>>>(G.n, wp, sh.k, pA, pB, q, x, r, f); ::sghsc::note_launch(); }
    SG_CHECK_LAUNCH();
    return SG_OK;
  };
  SG_TRY(capture_while(h, s, pre, body));
  if (dst_t == SG_F64)
    { k_scatter<T, double><<<shs.grid, shs.bdim, 0, s>>>(G.n, w, wp, shs.k, x, (double*)dst, ld_dst, fa.ctl); ::sghsc::note_launch(); }
  else
    { k_scatter<T, float><<<shs.grid, shs.bdim, 0, s>>>(G.n, w, wp, shs.k, x, (float*)dst, ld_dst, fa.ctl); ::sghsc::note_launch(); }
  SG_CHECK_LAUNCH();
  return SG_OK;
}

int inner_solve(sg_problem* h, int dtype, const void* src, int ld_src, int src_t, void* dst, int ld_dst, int dst_t,
                int w, const sg_prec_opts& o, cudaStream_t s) {
  SG_TRY(check_prec_opts(o));
  if (w <= 0) return SG_OK;
  if (o.m0 == SG_M0_VCYCLE && cluster_usable(h, dtype, w))
    return inner_solve_cluster(h, src, ld_src, src_t, dst, ld_dst, dst_t, w, o, s);
  SG_TRY(ensure_inner_work(h, dtype, std::max(w, h->wmax)));
  if (dtype == SG_F64) return inner_solve_t<double>(h, src, ld_src, src_t, dst, ld_dst, dst_t, w, o, s);
  return inner_solve_t<float>(h, src, ld_src, src_t, dst, ld_dst, dst_t, w, o, s);
}

// One V-cycle on the packed n x w block B into the packed block X: B is
// packed into the padded workspace, the cycle runs there, the result is
// unpacked into X.
template <typename T>
static int vcycle_packed(sg_problem* h, InnerWork& iw, const T* B, T* bpad, T* X, int w, const sg_prec_opts& o,
                         cudaStream_t s) {
  constexpr int N = VW<T>::N;
  const GridLevel& G = h->grids[0];
  const int wp = padded_width<T>(w);
  const Shape sh = make_shape(h, G.n, wp / N);
  { k_pack<T, T><<<sh.grid, sh.bdim, 0, s>>>(G.n, w, wp, sh.k, B, w, bpad); ::sghsc::note_launch(); }
  const T* res = nullptr;
  SG_TRY(vcycle<T>(h, iw, 0, bpad, (T*)iw.z, (T*)iw.zt, wp, o, s, nullptr, &res));
  { k_scatter<T, T><<<sh.grid, sh.bdim, 0, s>>>(G.n, w, wp, sh.k, res, X, w, nullptr); ::sghsc::note_launch(); }
  SG_CHECK_LAUNCH();
  return SG_OK;
}

// The mean-value preconditioner M_0 alone (one V-cycle, or D^{-1} with the
// diagonal M_0) on the w columns of a strided block: src, dst with leading
// dimensions lds, ldd, element type dtype on both sides.
template <typename T>
static int m0_apply_t(sg_problem* h, const T* src, int lds, T* dst, int ldd, int w, const sg_prec_opts& o,
                      cudaStream_t s) {
  constexpr int N = VW<T>::N;
  InnerWork& iw = sizeof(T) == 8 ? h->iw64 : h->iw32;
  const GridLevel& G = h->grids[0];
  const int wp = padded_width<T>(w);
  const Shape sh = make_shape(h, G.n, wp / N);
  { k_clear_done<<<1, 1024, 0, s>>>(iw.wcap, iw.done); ::sghsc::note_launch(); }
  { k_pack<T, T><<<sh.grid, sh.bdim, 0, s>>>(G.n, w, wp, sh.k, src, lds, (T*)iw.r); ::sghsc::note_launch(); }
  const T* res = nullptr;
  SG_TRY(vcycle<T>(h, iw, 0, (const T*)iw.r, (T*)iw.z, (T*)iw.zt, wp, o, s, nullptr, &res));
  { k_scatter<T, T><<<sh.grid, sh.bdim, 0, s>>>(G.n, w, wp, sh.k, res, dst, ldd, nullptr); ::sghsc::note_launch(); }
  SG_CHECK_LAUNCH();
  return SG_OK;
}

int m0_apply(sg_problem* h, int dtype, const void* src, int lds, void* dst, int ldd, int w, const sg_prec_opts& o,
             cudaStream_t s) {
  if (w <= 0) return SG_OK;
  SG_TRY(ensure_inner_work(h, dtype, std::max(w, h->wmax)));
  if (dtype == SG_F64) return m0_apply_t<double>(h, (const double*)src, lds, (double*)dst, ldd, w, o, s);
  return m0_apply_t<float>(h, (const float*)src, lds, (float*)dst, ldd, w, o, s);
}

int inner_vcycle(sg_problem* h, int dtype, const void* B, void* X, int w, const sg_prec_opts& o, cudaStream_t s) {
  SG_TRY(check_prec_opts(o));
  if (!h->mg_full || o.m0 != SG_M0_VCYCLE) {
    set_error("V-cycle: needs the whole multigrid hierarchy (power-of-two square mesh)");
    return SG_ERR_UNSUPPORTED;
  }
  SG_TRY(ensure_inner_work(h, dtype, std::max(w, h->wmax)));
  InnerWork& iw = dtype == SG_F64 ? h->iw64 : h->iw32;
  { k_clear_done<<<1, 1024, 0, s>>>(iw.wcap, iw.done); ::sghsc::note_launch(); }
  if (dtype == SG_F64) return vcycle_packed<double>(h, iw, (const double*)B, (double*)iw.r, (double*)X, w, o, s);
  return vcycle_packed<float>(h, iw, (const float*)B, (float*)iw.r, (float*)X, w, o, s);
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
static std::mutex g_static_scratch_mu;

// Device address of g_static_scratch on the current device (the name is only
// a host-side stand-in for the device array). A successful lookup is kept for
// the rest of the process; a failed one is not, so a later call retries it,
// and the failed call's error is taken off the runtime's error state so that
// it is not reported again by an unrelated launch check.
static int static_scratch(void** out) {
  int dev = 0;
  SG_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= STATIC_MAX_DEVICES) {
    set_error("sg_vcycle_apply_static: device ordinal %d not supported", dev);
    return SG_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_static_scratch_mu);
  if (!g_static_scratch_ptr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      set_error("sg_vcycle_apply_static: cudaGetSymbolAddress failed on device %d: %s", dev, cudaGetErrorString(e));
      return SG_ERR_CUDA;
    }
    g_static_scratch_ptr[dev] = ptr;
  }
  *out = g_static_scratch_ptr[dev];
  return SG_OK;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Bytes of V-cycle scratch for w columns (padded width wp): the done mask, the
// packed right-hand side and two iterates on the finest grid, and three blocks
// per coarser grid.
static size_t static_vcycle_bytes(const sg_problem* h, int wp, size_t es) {
  size_t b = align256((size_t)wp * sizeof(int));
  b += 3 * align256((size_t)h->grids[0].n * wp * es);
  for (size_t g = 1; g < h->grids.size(); ++g) b += 3 * align256((size_t)h->grids[g].n * wp * es);
  return b;
}

int vcycle_static(sg_problem* h, int dtype, const void* B, void* X, int w, const sg_prec_opts& o, cudaStream_t s) {
  SG_TRY(check_prec_opts(o));
  if (!h->mg_full || o.m0 != SG_M0_VCYCLE) {
    set_error("sg_vcycle_apply_static: no multigrid hierarchy (mesh missing or not a power-of-two square)");
    return SG_ERR_UNSUPPORTED;
  }
  const size_t es = dtype == SG_F64 ? 8 : 4;
  const int wp = dtype == SG_F64 ? padded_width<double>(w) : padded_width<float>(w);
  const size_t need = static_vcycle_bytes(h, wp, es);
  if (need > STATIC_SCRATCH_BYTES) {
    set_error("sg_vcycle_apply_static: %d columns of %d nodes need %zu bytes of scratch, above the fixed %zu",
              w, h->grids[0].n, need, STATIC_SCRATCH_BYTES);
    return SG_ERR_INVALID_ARG;
  }
  void* base = nullptr;
  SG_TRY(static_scratch(&base));
  unsigned char* p = (unsigned char*)base;
  InnerWork sw;  // views into the static array; nothing here allocates
  sw.wcap = wp;
  sw.esize = es;
  sw.done = (int*)p;
  p += align256((size_t)wp * sizeof(int));
  sw.r = p;
  p += align256((size_t)h->grids[0].n * wp * es);
  sw.z = p;
  p += align256((size_t)h->grids[0].n * wp * es);
  sw.zt = p;
  p += align256((size_t)h->grids[0].n * wp * es);
  const int G = (int)h->grids.size();
  sw.cb.assign(G, nullptr);
  sw.cx.assign(G, nullptr);
  sw.cxt.assign(G, nullptr);
  for (int g = 1; g < G; ++g) {
    const size_t bytes = align256((size_t)h->grids[g].n * wp * es);
    sw.cb[g] = p;
    p += bytes;
    sw.cx[g] = p;
    p += bytes;
    sw.cxt[g] = p;
    p += bytes;
  }
  // the kernels skip columns whose done flag is set: start from all zero
  SG_TRY_CUDA(cudaMemsetAsync(sw.done, 0, (size_t)wp * sizeof(int), s));
  if (dtype == SG_F64) return vcycle_packed<double>(h, sw, (const double*)B, (double*)sw.r, (double*)X, w, o, s);
  return vcycle_packed<float>(h, sw, (const float*)B, (float*)sw.r, (float*)X, w, o, s);
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
