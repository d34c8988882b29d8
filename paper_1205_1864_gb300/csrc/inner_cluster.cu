// K3 + K4 on chip: the batched inner PCG on A_0 with its V-cycle, one launch
// per solve, the whole multigrid hierarchy of a column group held in the
// shared memory of one thread-block cluster.
//
// Same method as the stand-alone kernels of inner.cu (Sec. 5: independent
// preconditioned CG loops on A_0 for the columns of a degree level; the
// V-cycle with weighted Jacobi, nu sweeps before and after, bilinear
// transfers and the Galerkin coarse operators of setup.cu as M_0), same
// per-column stopping rule, status bits and iteration counts. What differs is
// where the data lives:
//
// - A cluster of CLN = 8 CTAs (or 16, where that many are resident: half the
//   rows per CTA, for batches of at most 4 x the resident clusters) owns 4
//   columns (one float4 per node). Every grid with at least as many rows as
//   the cluster has CTAs is split into row strips, strip c on CTA c; the
//   smaller grids sit in CTA 0 alone. Each strip is stored with a ghost
//   row above and below and a ghost column left and right; ghosts outside the
//   grid stay zero, so every stencil phase is branch-free.
// - A phase that reads neighbours first copies the boundary rows it needs
//   from the neighbouring CTAs' shared memory (distributed shared memory)
//   into its ghost rows. Phases that depend on each other are separated by
//   cluster barriers; the grids held by CTA 0 alone use block barriers.
// - Per-column sums: the block's sum goes to a slot of its own (one slot per
//   kind of sum, so a slot is never rewritten while another CTA may read it);
//   after the cluster barrier every CTA adds the slots in rank order, so all
//   CTAs hold identical CG scalars and take the same loop decisions.
// - On the finest grid each thread owns up to FINE_ITEMS nodes, one below the
//   other (a stencil sweep rolls its 3 x 3 window down: 3 new loads per node),
//   and keeps their r and p in registers; the solution (x += alpha
//   p once per iteration) and q = A p of the last step go to a per-cluster
//   scratch in global memory (one coalesced float4 per node); the shared-memory
//   vectors there are the V-cycle iterate and its ping-pong partner.
//
// Eligibility (cluster_setup): a square hierarchy (power-of-two elements)
// whose shared-memory plan fits one CTA, at least one cluster resident, FP32.
// Anything else takes the stand-alone kernels.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdlib>

#include "sghsc_internal.cuh"
#include "vec.cuh"

namespace cg = cooperative_groups;

namespace sghsc {

constexpr int CLN = 8;          // CTAs per cluster (portable cluster size)
constexpr int CNT = 512;        // threads per CTA (128 registers each: no spills)
constexpr int CMAXG = 8;        // grids of the hierarchy (127 x 127 has 7)
constexpr int FINE_ITEMS = 4;   // finest-grid nodes per thread

// One grid of the hierarchy as laid out in every CTA's shared memory. Vector
// buffers are float4 [(rows + 2) x (nx + 2)] (padded: ghost rows and columns);
// the stencil holds the strip's own nodes [rows * nx][9]; the inverse diagonal
// is padded like the vectors (its ghost rows are needed by the fused first
// two sweeps). The finest grid has no b buffer and no inverse diagonal in
// shared memory (both are per-thread registers there).
struct CLevel {
  int nx, ny, rows, single;
  unsigned b, x, y, st, di;   // byte offsets into the dynamic shared memory
  const float* gst;           // stencil [n][9] in global memory
  const float* gdi;           // inverse diagonal [n]
};

struct CPlan {
  int G, gs;        // number of grids; first grid held by CTA 0 alone
  unsigned bytes;   // dynamic shared memory per CTA
  int maxcl;        // clusters resident at once (host side: one-wave rule)
  int fine_h;       // finest-grid rows per thread (a column segment of fine_h nodes)
  CLevel L[CMAXG];
};

struct CArgs {
  float om;
  int nu;
  double tol2;
  int maxit, fixed;
  int* status;
  long long* iacc;
  int* iters;   // per-column iteration counts out (global column index), or null
  float4* xs;   // solution scratch [cluster][n]: one float4 (4 columns) per node
  float4* qs;   // A p of the last step, same layout
};

namespace {

struct ColState {
  double rho, bb;
  int iters, done;
};

enum { RK_INIT = 0, RK_RHO, RK_PQ, RK_RR, RK_COUNT };

struct Own {
  int r0, nr;
};

__device__ __forceinline__ Own own_rows(const CLevel& l, int rank) {
  if (l.single) return Own{0, rank == 0 ? l.ny : 0};
  const int r0 = rank * l.rows;
  return Own{r0, max(0, min(l.ny - r0, l.rows))};
}

// padded index of local row ly (-1 .. rows) and column x (-1 .. nx)
__device__ __forceinline__ int pidx(const CLevel& l, int ly, int x) { return (ly + 1) * (l.nx + 2) + x + 1; }

template <typename T>
__device__ __forceinline__ T* sp(unsigned char* sm, unsigned off) {
  return reinterpret_cast<T*>(sm + off);
}

__device__ __forceinline__ float4 f4(float a) { return make_float4(a, a, a, a); }

__device__ __forceinline__ void fma4(float4& acc, float a, const float4& v) {
  acc.x = fmaf(a, v.x, acc.x);
  acc.y = fmaf(a, v.y, acc.y);
  acc.z = fmaf(a, v.z, acc.z);
  acc.w = fmaf(a, v.w, acc.w);
}

__device__ __forceinline__ float4 add4(const float4& a, const float4& b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

__device__ __forceinline__ float4 sub4(const float4& a, const float4& b) {
  return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}

// acc += a * b componentwise (fused)
__device__ __forceinline__ void dot4(float4& acc, const float4& a, const float4& b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.y = fmaf(a.y, b.y, acc.y);
  acc.z = fmaf(a.z, b.z, acc.z);
  acc.w = fmaf(a.w, b.w, acc.w);
}

__device__ __forceinline__ float comp(const float4& v, int u) {
  return u == 0 ? v.x : u == 1 ? v.y : u == 2 ? v.z : v.w;
}

// sum_j a_ij v_j over the 9-point stencil s9 of the node at padded index c
// (row length W of the padded buffer)
__device__ __forceinline__ float4 apply9(const float* __restrict__ s9, const float4* v, int W, int c) {
  float4 acc = f4(0.f);
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) fma4(acc, s9[(dy + 1) * 3 + (dx + 1)], v[c + dy * W + dx]);
  return acc;
}

// 4-byte global -> shared copy without a register round trip (cp.async);
// copy_async_wait completes this thread's copies.
__device__ __forceinline__ void copy_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}

// 16-byte copy (both addresses 16-byte aligned)
__device__ __forceinline__ void copy_async16(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

// cnt floats global -> shared: 16-byte copies where the two addresses share
// their alignment (a 4-byte head up to the boundary and a 4-byte tail), 4-byte
// copies otherwise; the block's threads share the work.
__device__ __forceinline__ void stage_floats(float* dst, const float* src, int cnt) {
  if ((((size_t)dst ^ (size_t)src) & 15) == 0) {
    const int head = min(cnt, (int)(((16 - ((size_t)dst & 15)) & 15) / 4));
    const int body = (cnt - head) / 4;
    for (int i = threadIdx.x; i < head; i += blockDim.x) copy_async4(dst + i, src + i);
    for (int i = threadIdx.x; i < body; i += blockDim.x) copy_async16(dst + head + 4 * i, src + head + 4 * i);
    for (int i = head + 4 * body + threadIdx.x; i < cnt; i += blockDim.x) copy_async4(dst + i, src + i);
  } else {
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) copy_async4(dst + i, src + i);
  }
}

__device__ __forceinline__ void copy_async_wait() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Store v at own node (ly, x) of buffer off of grid l; on a distributed grid
// also into the ghost row of the neighbouring strip that sees this node (the
// first own row is the ghost row below of CTA rank - 1, the last one the ghost
// row above of CTA rank + 1). The next cluster barrier publishes both, so a
// phase never reads the buffer it writes and needs no copy step of its own.
__device__ __forceinline__ void put(const cg::cluster_group& cl, unsigned char* sm, const CLevel& l, unsigned off,
                                    int rank, const Own& o, int ly, int x, const float4& v) {
  float4* b = sp<float4>(sm, off);
  b[pidx(l, ly, x)] = v;
  if (l.single) return;
  if (ly == 0 && o.r0 > 0) cl.map_shared_rank(b, rank - 1)[pidx(l, l.rows, x)] = v;
  if (ly == o.nr - 1 && o.r0 + o.nr < l.ny) cl.map_shared_rank(b, rank + 1)[pidx(l, -1, x)] = v;
}

// Compiler scheduling fence: memory accesses are not moved across it. Placed
// between the finest-grid nodes of a thread and between the parts of the
// prolongation, so not all their loads are in flight at once (their
// registers would spill).
__device__ __forceinline__ void item_fence() { asm volatile("" ::: "memory"); }

// Interpolation weight of coarse patch entry a (0..2: coarse offset a - 1
// from floor((f - 1) / 2)) at the fine point f + d (d = -1..1), for a fine
// coordinate f of parity odd. Coarse node X sits on fine node 2X + 1, so an
// odd fine point takes its coarse node with weight 1 and an even one the two
// coarse nodes beside it with weight 1/2 (bilinear interpolation is the
// product of the x and y weights).
__device__ __forceinline__ float tw(bool odd, int d, int a) {
  if (odd) return d < 0 ? (a < 2 ? 0.5f : 0.f) : d == 0 ? (a == 1 ? 1.f : 0.f) : (a > 0 ? 0.5f : 0.f);
  return d < 0 ? (a == 1 ? 1.f : 0.f) : d == 0 ? (a > 0 ? 0.5f : 0.f) : (a == 2 ? 1.f : 0.f);
}

// The coarse correction at a fine node (y, x) with stencil s9: pc = (P xc) at
// the node and apc = sum_j a_ij (P xc)_j over its stencil, from the 3 x 3
// coarse patch around padded coarse index cc = (floor((y-1)/2), floor((x-1)/2)).
// A(P xc) = sum_{a,c} K[a][c] xc[a][c] with K = Wy^T S Wx (the x and y
// interpolation weights of the three fine rows / columns). Patch entries whose
// weights are all zero (row a = 0 for even y, column 0 for even x) would lie
// outside the padded strip at the grid edge: they read entry 1 instead, with
// weight zero.
__device__ __forceinline__ void coarse_corr(const float* __restrict__ s9, const float4* XC, int Wc, int cc, bool oy,
                                            bool ox, float4& apc, float4& pc) {
  float t1[3][3];   // t1[dy][c] = sum_dx s[dy][dx] wx(dx, c)
#pragma unroll
  for (int dy = 0; dy < 3; ++dy)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      t1[dy][c] = s9[dy * 3 + 0] * tw(ox, -1, c) + s9[dy * 3 + 1] * tw(ox, 0, c) + s9[dy * 3 + 2] * tw(ox, 1, c);
  apc = f4(0.f);
  pc = f4(0.f);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    item_fence();
    const int ar = (oy || a > 0) ? a : 1;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int cr = (ox || c > 0) ? c : 1;
      const float K = tw(oy, -1, a) * t1[0][c] + tw(oy, 0, a) * t1[1][c] + tw(oy, 1, a) * t1[2][c];
      const float4 v = XC[cc + (ar - 1) * Wc + (cr - 1)];
      fma4(apc, K, v);
      fma4(pc, tw(oy, 0, a) * tw(ox, 0, c), v);
    }
  }
}

// x + om d (b - A x) at the node of padded index c
__device__ __forceinline__ float4 jacobi_node(const float* __restrict__ s9, const float4* X, int W, int c,
                                              const float4& b, float d, float om) {
  const float4 ax = apply9(s9, X, W, c);
  const float4 xv = X[c];
  const float dd = om * d;
  return make_float4(fmaf(dd, b.x - ax.x, xv.x), fmaf(dd, b.y - ax.y, xv.y), fmaf(dd, b.z - ax.z, xv.z),
                     fmaf(dd, b.w - ax.w, xv.w));
}

// x' = x + P xc, then x' + om d (b - A x') at fine node (y, x) of padded index c
__device__ __forceinline__ float4 prolong_jacobi_node(const float* __restrict__ s9, const float4* X, int W, int c,
                                                      const float4& b, float d, float om, const float4* XC,
                                                      int Wc, int cc, bool oy, bool ox) {
  const float4 ax = apply9(s9, X, W, c);
  item_fence();
  float4 apc, pc;
  coarse_corr(s9, XC, Wc, cc, oy, ox, apc, pc);
  const float4 xv = add4(X[c], pc);
  const float dd = om * d;
  return make_float4(fmaf(dd, b.x - (ax.x + apc.x), xv.x), fmaf(dd, b.y - (ax.y + apc.y), xv.y),
                     fmaf(dd, b.z - (ax.z + apc.z), xv.z), fmaf(dd, b.w - (ax.w + apc.w), xv.w));
}

// padded index, in the coarse grid lc as held by CTA rank, of the coarse patch
// centre of fine node (y, x)
__device__ __forceinline__ int patch_centre(const CLevel& lc, int rank, int y, int x) {
  const int r0c = lc.single ? 0 : rank * lc.rows;
  return pidx(lc, ((y - 1) >> 1) - r0c, (x - 1) >> 1);
}

// bc = P^T R on the coarse rows Y whose centre fine row 2Y + 1 is one of this
// CTA's rows of grid l (the fine rows 2Y and 2Y + 2 are own rows or ghosts),
// stored into the coarse right-hand side of the CTA that owns row Y (and the
// ghost rows of its neighbours, as put() does). Weights
// 1 (centre), 1/2 (edge) and 1/4 (corner): the transpose of the bilinear
// interpolation.
// R: the residual as padded rows of this CTA (local row 0 = grid row o.r0),
// in shared memory or, on the finest grid of the wide solver, in global memory.
__device__ void restrict_rows(const cg::cluster_group& cl, unsigned char* sm, const CLevel& l, const Own& o,
                              const float4* R, const CLevel& lc, int rank) {
  const int top = o.r0 + o.nr - 2;
  if (o.nr == 0 || top < 0) return;
  const int ylo = o.r0 / 2, yhi = min(top / 2, lc.ny - 1);
  const int W = l.nx + 2;
  const int items = (yhi - ylo + 1) * lc.nx;
  for (int i = threadIdx.x; i < items; i += blockDim.x) {
    const int Y = ylo + i / lc.nx, X = i % lc.nx;
    const int c = pidx(l, 2 * Y + 1 - o.r0, 2 * X + 1);
    float4 acc = f4(0.f);
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) fma4(acc, (dy == 0 ? 1.f : 0.5f) * (dx == 0 ? 1.f : 0.5f), R[c + dy * W + dx]);
    const int ow = lc.single ? 0 : Y / lc.rows, lr = Y - ow * lc.rows;
    float4* Bc = sp<float4>(sm, lc.b);
    cl.map_shared_rank(Bc, ow)[pidx(lc, lr, X)] = acc;
    if (!lc.single) {
      if (lr == 0 && ow > 0) cl.map_shared_rank(Bc, ow - 1)[pidx(lc, lc.rows, X)] = acc;
      if (lr == min(lc.rows, lc.ny - ow * lc.rows) - 1 && Y + 1 < lc.ny)
        cl.map_shared_rank(Bc, ow + 1)[pidx(lc, -1, X)] = acc;
    }
  }
}

// Fixed-order block sum of the per-thread partials v into *slot (written by
// thread 0): warp butterflies, then warp 0 over the warp sums.
__device__ void block_sum4(float4 v, float4* wred, float4* slot) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    v.z += __shfl_xor_sync(0xffffffffu, v.z, o);
    v.w += __shfl_xor_sync(0xffffffffu, v.w, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) wred[wid] = v;
  __syncthreads();
  if (wid == 0) {
    float4 s = lane < (int)(blockDim.x >> 5) ? wred[lane] : f4(0.f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
      s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
      s.z += __shfl_xor_sync(0xffffffffu, s.z, o);
      s.w += __shfl_xor_sync(0xffffffffu, s.w, o);
    }
    if (lane == 0) *slot = s;
  }
}

// Shared state of one CTA: per-column CG scalars (identical in all CTAs of the
// cluster), the FP32 step lengths the kernels use, the loop flag, and the
// reduction scratch.
struct CShared {
  float4 wred[CNT / 32];
  float4 slot[RK_COUNT];
  ColState cs[4];
  float alpha[4], beta[4];
  int active;
};

// After the cluster barrier that follows the slot writes: lanes 0..3 of warp 0
// each add the CTAs' slots in rank order and update their column (the
// scalar updates of the stand-alone finaliser: FP64 from the FP32 totals);
// rank 0 reports status bits and iteration counts. Ends with a block barrier.
// NCT: CTAs per cluster, 0 = read at run time (a kernel launched with either size).
template <int NCT>
__device__ void col_step(const cg::cluster_group& cl, CShared& S, int kind, const CArgs& a, int rank) {
  const int lane = threadIdx.x;
  if (lane < 4) {
    float4 tot = f4(0.f);
    const int nct = NCT > 0 ? NCT : (int)cl.num_blocks();   // 8 or 16
    for (int h = 0; h < nct; h += 8) {   // 8 remote loads in flight, then the sums in rank order
      float4 v[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) v[r] = *cl.map_shared_rank(&S.slot[kind], h + r);
#pragma unroll
      for (int r = 0; r < 8; ++r) tot = add4(tot, v[r]);
    }
    const double s = (double)comp(tot, lane);
    const bool report = rank == 0;
    ColState c = S.cs[lane];
    if (kind == RK_INIT) {
      c.bb = s;
      c.done = !(s > 0.0);
      c.iters = 0;
      S.beta[lane] = 0.f;
    } else if (!c.done) {
      if (kind == RK_RHO) {
        const double beta = c.iters == 0 ? 0.0 : s / c.rho;
        S.beta[lane] = (float)beta;
        c.rho = s;
      } else if (kind == RK_PQ) {
        double alpha = 0.0;
        if (!(s > 0.0)) {
          if (report) atomicOr(a.status, ST_INNER_NOT_SPD);
          c.done = 1;
        } else {
          alpha = c.rho / s;
        }
        S.alpha[lane] = (float)alpha;
      } else {
        const int it = ++c.iters;
        bool fin;
        if (a.fixed > 0) {
          fin = it >= a.fixed;
        } else {
          fin = s <= a.tol2 * c.bb;
          if (!fin && it >= a.maxit) {
            fin = true;
            if (report) atomicOr(a.status, ST_INNER_MAXIT);
          }
        }
        if (!(s == s)) {   // non-finite residual: stop the column and flag it
          fin = true;
          if (report) atomicOr(a.status, ST_INNER_NOT_SPD);
        }
        c.done = fin;
        if (fin && report) {
          atomicAdd((unsigned long long*)&a.iacc[0], (unsigned long long)it);
          atomicMax(&a.iacc[1], (long long)it);
        }
      }
    }
    S.cs[lane] = c;
  }
  __syncwarp();
  if (lane == 0) S.active = !(S.cs[0].done && S.cs[1].done && S.cs[2].done && S.cs[3].done);
  __syncthreads();
}

// Sum of the per-thread partials v over the cluster into the column scalars
// (slot kind), then the column update: block sum, cluster barrier, col_step.
template <int NCT>
__device__ __forceinline__ void cluster_reduce(const cg::cluster_group& cl, CShared& S, int kind, const float4& v,
                                               const CArgs& a, int rank) {
  block_sum4(v, S.wred, &S.slot[kind]);
  cluster_sync_all();
  col_step<NCT>(cl, S, kind, a, rank);
}


// Buffer holding the iterate of grid l after its pre-smoothing (the smoother
// alternates between x and y: max(0, nu - 2) exchanges) ...
__device__ __forceinline__ unsigned after_down(const CLevel& l, int nu) { return (max(0, nu - 2) & 1) ? l.y : l.x; }

// ... and after its post-smoothing (nu more); the coarsest grid is solved into x.
__device__ __forceinline__ unsigned final_buf(const CLevel& l, bool coarsest, int nu) {
  if (coarsest) return l.x;
  return ((max(0, nu - 2) + nu) & 1) ? l.y : l.x;
}

// blk: a grid held by CTA 0 alone (block barrier), else the cluster barrier
__device__ __forceinline__ void level_sync(bool blk) {
  if (blk) __syncthreads();
  else cluster_sync_all();
}

// f(i, ly, x) for this CTA's nodes of grid l (i: own node index)
template <typename F>
__device__ __forceinline__ void for_own(const CLevel& l, const Own& o, F f) {
  const int n = o.nr * l.nx;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int ly = i / l.nx;
    f(i, ly, i - ly * l.nx);
  }
}

// Restriction side of the V-cycle on a coarse grid g (right-hand side in its
// b buffer, zero initial iterate): nu sweeps, the residual, and its
// restriction into grid g + 1. A grid held by CTA 0 alone is run by CTA 0
// with block barriers (one copy of the code serves both kinds of grid: the
// kernel's phases each run once per iteration, and its size decides how much
// of it the instruction cache keeps).
__device__ __noinline__ void level_down(const cg::cluster_group& cl, unsigned char* sm, const CLevel* L, int g,
                                        int rank, int nu, float om) {
  const CLevel& l = L[g];
  const bool blk = l.single;
  const Own o = own_rows(l, rank);
  const int W = l.nx + 2;
  const float* ST = sp<float>(sm, l.st);
  const float* DI = sp<float>(sm, l.di);
  const float4* B = sp<float4>(sm, l.b);
  unsigned xo = l.x, yo = l.y;
  if (nu >= 2) {
    // the first two sweeps in one pass: x1 = om D^-1 b at the 9 neighbours,
    // x2 = x1 + om D^-1 (b - A x1)
    for_own(l, o, [&](int i, int ly, int x) {
      const int c = pidx(l, ly, x);
      const float* s9 = ST + i * 9;
      float4 ax1 = f4(0.f);
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const int j = c + dy * W + dx;
          fma4(ax1, s9[(dy + 1) * 3 + (dx + 1)] * DI[j], B[j]);
        }
      const float dd = om * DI[c];
      const float4 b = B[c];
      put(cl, sm, l, xo, rank, o, ly, x,
          make_float4(dd * b.x + dd * (b.x - om * ax1.x), dd * b.y + dd * (b.y - om * ax1.y),
                      dd * b.z + dd * (b.z - om * ax1.z), dd * b.w + dd * (b.w - om * ax1.w)));
    });
    level_sync(blk);
    for (int s = 2; s < nu; ++s) {
      const float4* Xi = sp<float4>(sm, xo);
      for_own(l, o, [&](int i, int ly, int x) {
        const int c = pidx(l, ly, x);
        put(cl, sm, l, yo, rank, o, ly, x, jacobi_node(ST + i * 9, Xi, W, c, B[c], DI[c], om));
      });
      level_sync(blk);
      const unsigned t = xo; xo = yo; yo = t;
    }
  } else {
    for_own(l, o, [&](int, int ly, int x) {
      const int c = pidx(l, ly, x);
      const float dd = om * DI[c];
      const float4 b = B[c];
      put(cl, sm, l, xo, rank, o, ly, x, make_float4(dd * b.x, dd * b.y, dd * b.z, dd * b.w));
    });
    level_sync(blk);
  }
  // residual b - A x into the other buffer, then its restriction
  {
    const float4* X = sp<float4>(sm, xo);
    for_own(l, o, [&](int i, int ly, int x) {
      const int c = pidx(l, ly, x);
      put(cl, sm, l, yo, rank, o, ly, x, sub4(B[c], apply9(ST + i * 9, X, W, c)));
    });
  }
  level_sync(blk);
  restrict_rows(cl, sm, l, o, sp<float4>(sm, yo), L[g + 1], rank);
  level_sync(blk);
}

// Prolongation side on a coarse grid g: the correction from grid g + 1 with
// the first post-smoothing sweep in one pass, then nu - 1 more sweeps.
__device__ __noinline__ void level_up(const cg::cluster_group& cl, unsigned char* sm, const CLevel* L, int g, int G,
                                      int rank, int nu, float om) {
  const CLevel& l = L[g];
  const bool blk = l.single;
  const CLevel& lc = L[g + 1];
  const Own o = own_rows(l, rank);
  const int W = l.nx + 2, Wc = lc.nx + 2;
  const float* ST = sp<float>(sm, l.st);
  const float* DI = sp<float>(sm, l.di);
  const float4* B = sp<float4>(sm, l.b);
  unsigned xo = after_down(l, nu);
  unsigned yo = xo == l.x ? l.y : l.x;
  {
    const float4* X = sp<float4>(sm, xo);
    const float4* XC = sp<float4>(sm, final_buf(lc, g + 1 == G - 1, nu));
    for_own(l, o, [&](int i, int ly, int x) {
      const int c = pidx(l, ly, x), y = o.r0 + ly;
      put(cl, sm, l, yo, rank, o, ly, x,
          prolong_jacobi_node(ST + i * 9, X, W, c, B[c], DI[c], om, XC, Wc, patch_centre(lc, rank, y, x), y & 1,
                              x & 1));
    });
  }
  level_sync(blk);
  {
    const unsigned t = xo; xo = yo; yo = t;
  }
  for (int s = 1; s < nu; ++s) {
    const float4* Xi = sp<float4>(sm, xo);
    for_own(l, o, [&](int i, int ly, int x) {
      const int c = pidx(l, ly, x);
      put(cl, sm, l, yo, rank, o, ly, x, jacobi_node(ST + i * 9, Xi, W, c, B[c], DI[c], om));
    });
    level_sync(blk);
    const unsigned t = xo; xo = yo; yo = t;
  }
}

// The grids gs .. G-1 held by CTA 0: the rest of the V-cycle with block
// barriers; the coarsest grid (one node) is solved exactly, x = D^-1 b. The
// result on grid gs is then copied into the other CTAs (the prolongation onto
// grid gs - 1 reads it everywhere); the caller's cluster barrier publishes it.
__device__ void block_levels(const cg::cluster_group& cl, unsigned char* sm, const CLevel* L, int gs, int G, int nu,
                             float om) {
  for (int g = gs; g < G - 1; ++g) level_down(cl, sm, L, g, 0, nu, om);
  {
    const CLevel& l = L[G - 1];
    const Own o = own_rows(l, 0);
    const float* DI = sp<float>(sm, l.di);
    const float4* B = sp<float4>(sm, l.b);
    float4* X = sp<float4>(sm, l.x);
    for_own(l, o, [&](int, int ly, int x) {
      const int c = pidx(l, ly, x);
      const float d = DI[c];
      const float4 b = B[c];
      X[c] = make_float4(d * b.x, d * b.y, d * b.z, d * b.w);
    });
    __syncthreads();
  }
  for (int g = G - 2; g >= gs; --g) level_up(cl, sm, L, g, G, 0, nu, om);
  // each other CTA receives the rows of grid gs that the correction of its own
  // rows y of grid gs - 1 reads: patch centres (y - 1) / 2, one row either side
  const CLevel& l = L[gs];
  const CLevel& lf = L[gs - 1];
  float4* v = sp<float4>(sm, final_buf(l, gs == G - 1, nu));
  // (at most K = rows / 2 + 4 rows per CTA; one flat loop over all of them)
  const int W = l.nx + 2, nct = (int)cl.num_blocks(), K = lf.rows / 2 + 4;
  for (int i = threadIdx.x; i < (nct - 1) * K * W; i += blockDim.x) {
    const int r = 1 + i / (K * W), q = i % (K * W);
    const Own of = own_rows(lf, r);
    const int lo = max(0, ((of.r0 - 1) >> 1) - 1), hi = min(l.ny - 1, ((of.r0 + of.nr - 2) >> 1) + 1);
    const int y = lo + q / W;
    if (of.nr > 0 && y <= hi) {
      const int j = (y + 1) * W + q % W;
      cl.map_shared_rank(v, r)[j] = v[j];
    }
  }
}

// The finest-grid stencil sweep of one thread over its fn nodes (fy0 + k, fx),
// k = 0 .. fn-1, one below the other: the 3 x 3 window of X around the node
// rolls down one row per node, so a node costs 3 new loads instead of 9.
// f(k, c, ax, xc) receives the padded index, (A X) and X at node k.
template <typename F>
__device__ __forceinline__ void fine_sweep(const float* __restrict__ ST, const float4* X, int W, int nx, int fy0,
                                           int fx, int fn, F f) {
  if (fn <= 0) return;
  const int c0 = (fy0 + 1) * W + fx + 1;
  float4 w0[3], w1[3], w2[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    w0[d] = X[c0 - W + d - 1];
    w1[d] = X[c0 + d - 1];
  }
#pragma unroll
  for (int k = 0; k < FINE_ITEMS; ++k) {
    if (k >= fn) break;
    const int c = c0 + k * W;
#pragma unroll
    for (int d = 0; d < 3; ++d) w2[d] = X[c + W + d - 1];
    const float* s9 = ST + ((fy0 + k) * nx + fx) * 9;
    float4 ax = f4(0.f);
#pragma unroll
    for (int d = 0; d < 3; ++d) fma4(ax, s9[d], w0[d]);
#pragma unroll
    for (int d = 0; d < 3; ++d) fma4(ax, s9[3 + d], w1[d]);
#pragma unroll
    for (int d = 0; d < 3; ++d) fma4(ax, s9[6 + d], w2[d]);
    f(k, c, ax, w1[1]);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      w0[d] = w1[d];
      w1[d] = w2[d];
    }
  }
}

// One column group's whole inner solve: gather, PCG iterations with the
// V-cycle, scatter. Grid: 8 or 16 CTAs per 4 columns, clusters of that size.
template <typename TS, typename TD>
__global__ void __launch_bounds__(CNT, 1)
    k_inner_cluster(const CPlan P, const TS* __restrict__ src, int lds, TD* __restrict__ dst, int ldd, int w,
                    const CArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ CLevel L[CMAXG];
  __shared__ CShared S;
  const cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int cid = (int)(blockIdx.x / cl.num_blocks());   // column group (clusters of 8 or 16)
  const int col0 = cid * 4;
  const int G = P.G, gs = P.gs, nu = a.nu;
  const float om = a.om;

  // ---- set-up: grid table; own-row stencils (asynchronous copies, in
  // flight during the rest of the set-up); zeroed vectors and diagonals
  // (ghosts outside the grids stay zero); diagonals with their ghost rows
#pragma unroll
  for (int g = 0; g < CMAXG; ++g)
    if ((int)threadIdx.x == g) L[g] = P.L[g];
  if (threadIdx.x < 4) {
    S.cs[threadIdx.x] = ColState{0.0, 0.0, 0, 1};
    S.alpha[threadIdx.x] = 0.f;
    S.beta[threadIdx.x] = 0.f;
  }
  __syncthreads();
  for (int g = 0; g < G; ++g) {
    const CLevel& l = L[g];
    const Own o = own_rows(l, rank);
    if (o.nr == 0) continue;
    stage_floats(sp<float>(sm, l.st), l.gst + (size_t)o.r0 * l.nx * 9, o.nr * l.nx * 9);
  }
  for (int g = 0; g < G; ++g) {
    const CLevel& l = L[g];
    const unsigned lo = g > 0 ? l.b : l.x;
    const unsigned end = g + 1 < G ? L[g + 1].b : P.bytes;
    float4* z = reinterpret_cast<float4*>(sm);
    for (int i = (int)(lo / 16) + threadIdx.x; i < (int)(l.st / 16); i += CNT) z[i] = f4(0.f);
    if (g > 0)
      for (int i = (int)(l.di / 16) + threadIdx.x; i < (int)(end / 16); i += CNT) z[i] = f4(0.f);
  }
  __syncthreads();
  for (int g = 1; g < G; ++g) {
    const CLevel& l = L[g];
    const Own o = own_rows(l, rank);
    if (o.nr == 0) continue;
    float* di = sp<float>(sm, l.di);
    const int lo = max(o.r0 - 1, 0) - o.r0, hi = min(o.r0 + o.nr + 1, l.ny) - o.r0;
    for (int i = threadIdx.x; i < (hi - lo) * l.nx; i += CNT) {
      const int ly = lo + i / l.nx, x = i % l.nx;
      copy_async4(di + pidx(l, ly, x), l.gdi + (size_t)(o.r0 + ly) * l.nx + x);
    }
  }

  // ---- finest grid. Thread t owns column fx = t mod nx0 of the rows fy0 ..
  // fy0 + fn - 1 (fy0 = fine_h (t div nx0)): vertically adjacent nodes, so a
  // stencil sweep rolls its window down (fine_sweep). r = b, x = 0, p = 0;
  // ||b||^2; the first smoothing sweep from zero (om D^-1 r) into the iterate.
  const CLevel& L0 = L[0];
  const Own o0 = own_rows(L0, rank);
  const int nx0 = L0.nx, W0 = nx0 + 2;
  const int fx = threadIdx.x % nx0, fy0 = P.fine_h * ((int)threadIdx.x / nx0);
  const int fn = (int)threadIdx.x < (CNT / nx0) * nx0 ? max(0, min(P.fine_h, o0.nr - fy0)) : 0;
  const float* ST0 = sp<float>(sm, L0.st);
  float4 r[FINE_ITEMS], po[FINE_ITEMS];   // the solution accumulates in a.xs
  float d0[FINE_ITEMS];
  // this CTA's nodes of the cluster's solution and A p scratch (recomputed where used)
#define XG (a.xs + (size_t)cid * P.L[0].nx * P.L[0].ny + (size_t)o0.r0 * nx0)
#define QG (a.qs + (size_t)cid * P.L[0].nx * P.L[0].ny + (size_t)o0.r0 * nx0)
#define FI(k) ((fy0 + (k)) * nx0 + fx)
  unsigned zo = L0.x, so = L0.y;
  float4 part = f4(0.f);
#pragma unroll
  for (int k = 0; k < FINE_ITEMS; ++k) {
    r[k] = f4(0.f);
    po[k] = f4(0.f);
    d0[k] = 0.f;
    if (k < fn) {
      const int i = FI(k);
      const size_t node = (size_t)o0.r0 * nx0 + i;
      float v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = col0 + u < w ? (float)src[node * lds + col0 + u] : 0.f;
      XG[i] = f4(0.f);
      r[k] = make_float4(v[0], v[1], v[2], v[3]);
      d0[k] = L0.gdi[node];
      dot4(part, r[k], r[k]);
      const float dd = om * d0[k];
      put(cl, sm, L0, zo, rank, o0, fy0 + k, fx, make_float4(dd * v[0], dd * v[1], dd * v[2], dd * v[3]));
    }
  }
  copy_async_wait();
  cluster_reduce<0>(cl, S, RK_INIT, part, a, rank);

  const int cap = (a.fixed > 0 ? a.fixed : a.maxit) + 1;
  for (int it = 0; it < cap && S.active; ++it) {
    // ---- V-cycle, finest grid down: sweeps 2..nu, residual, restriction
    for (int s = 1; s < nu; ++s) {
      fine_sweep(ST0, sp<float4>(sm, zo), W0, nx0, fy0, fx, fn, [&](int k, int, const float4& ax, const float4& xc) {
        const float dd = om * d0[k];
        put(cl, sm, L0, so, rank, o0, fy0 + k, fx,
            make_float4(fmaf(dd, r[k].x - ax.x, xc.x), fmaf(dd, r[k].y - ax.y, xc.y), fmaf(dd, r[k].z - ax.z, xc.z),
                        fmaf(dd, r[k].w - ax.w, xc.w)));
      });
      cluster_sync_all();
      const unsigned t = zo; zo = so; so = t;
    }
    fine_sweep(ST0, sp<float4>(sm, zo), W0, nx0, fy0, fx, fn, [&](int k, int, const float4& ax, const float4&) {
      put(cl, sm, L0, so, rank, o0, fy0 + k, fx, sub4(r[k], ax));
    });
    cluster_sync_all();
    restrict_rows(cl, sm, L0, o0, sp<float4>(sm, so), L[1], rank);
    cluster_sync_all();
    // ---- coarse grids
    for (int g = 1; g < gs; ++g) level_down(cl, sm, L, g, rank, nu, om);
    if (rank == 0) block_levels(cl, sm, L, gs, G, nu, om);
    cluster_sync_all();
    for (int g = gs - 1; g >= 1; --g) level_up(cl, sm, L, g, G, rank, nu, om);
    // ---- finest grid up: correction + sweep, nu - 1 more sweeps; the last
    // one also sums r . z
    const float4* XC = sp<float4>(sm, final_buf(L[1], G == 2, nu));
    const int Wc = L[1].nx + 2;
    for (int s = 1; s <= nu; ++s) {
      part = f4(0.f);
      fine_sweep(ST0, sp<float4>(sm, zo), W0, nx0, fy0, fx, fn, [&](int k, int, const float4& ax, const float4& xc) {
        const float dd = om * d0[k];
        float4 v;
        if (s == 1) {
          const int y = o0.r0 + fy0 + k;
          float4 apc, pc;
          coarse_corr(ST0 + FI(k) * 9, XC, Wc, patch_centre(L[1], rank, y, fx), y & 1, fx & 1, apc, pc);
          const float4 xv = add4(xc, pc);
          v = make_float4(fmaf(dd, r[k].x - (ax.x + apc.x), xv.x), fmaf(dd, r[k].y - (ax.y + apc.y), xv.y),
                          fmaf(dd, r[k].z - (ax.z + apc.z), xv.z), fmaf(dd, r[k].w - (ax.w + apc.w), xv.w));
        } else {
          v = make_float4(fmaf(dd, r[k].x - ax.x, xc.x), fmaf(dd, r[k].y - ax.y, xc.y), fmaf(dd, r[k].z - ax.z, xc.z),
                          fmaf(dd, r[k].w - ax.w, xc.w));
        }
        put(cl, sm, L0, so, rank, o0, fy0 + k, fx, v);
        dot4(part, r[k], v);
      });
      if (s == nu) cluster_reduce<0>(cl, S, RK_RHO, part, a, rank);
      else cluster_sync_all();
      const unsigned t = zo; zo = so; so = t;
    }
    // ---- p = z + beta p (registers), q = A p = A z + beta q_old (linearity:
    // the z of this step is complete with its ghost rows, so no p_new buffer
    // and no extra phase), p . q; q kept in registers and in the scratch
    float4 qv[FINE_ITEMS];
    {
      const float4 bt = make_float4(S.beta[0], S.beta[1], S.beta[2], S.beta[3]);
      float4* qg = QG;
#pragma unroll
      for (int k = 0; k < FINE_ITEMS; ++k) qv[k] = (it > 0 && k < fn) ? qg[FI(k)] : f4(0.f);
      part = f4(0.f);
      fine_sweep(ST0, sp<float4>(sm, zo), W0, nx0, fy0, fx, fn, [&](int k, int, const float4& az, const float4& z) {
        po[k] = make_float4(fmaf(bt.x, po[k].x, z.x), fmaf(bt.y, po[k].y, z.y), fmaf(bt.z, po[k].z, z.z),
                            fmaf(bt.w, po[k].w, z.w));
        qv[k] = make_float4(fmaf(bt.x, qv[k].x, az.x), fmaf(bt.y, qv[k].y, az.y), fmaf(bt.z, qv[k].z, az.z),
                            fmaf(bt.w, qv[k].w, az.w));
        dot4(part, po[k], qv[k]);
        qg[FI(k)] = qv[k];
      });
    }
    cluster_reduce<0>(cl, S, RK_PQ, part, a, rank);
    // ---- x += alpha p, r -= alpha q on the unfinished columns; r . r; the
    // next V-cycle's first sweep om D^-1 r
    {
      const float al0 = S.alpha[0], al1 = S.alpha[1], al2 = S.alpha[2], al3 = S.alpha[3];
      const bool dn0 = S.cs[0].done, dn1 = S.cs[1].done, dn2 = S.cs[2].done, dn3 = S.cs[3].done;
      const bool up0 = !dn0 && col0 < w, up1 = !dn1 && col0 + 1 < w, up2 = !dn2 && col0 + 2 < w,
                 up3 = !dn3 && col0 + 3 < w;
      // x += alpha p in the scratch (coalesced float4 per node; the loads
      // first, so they are in flight together)
      float4 xv[FINE_ITEMS];
      float4* xg = XG;
#pragma unroll
      for (int k = 0; k < FINE_ITEMS; ++k)
        if (k < fn) xv[k] = xg[FI(k)];
      part = f4(0.f);
#pragma unroll
      for (int k = 0; k < FINE_ITEMS; ++k) {
        if (k >= fn) break;
        float4 v = xv[k];
        if (up0) v.x = fmaf(al0, po[k].x, v.x);
        if (up1) v.y = fmaf(al1, po[k].y, v.y);
        if (up2) v.z = fmaf(al2, po[k].z, v.z);
        if (up3) v.w = fmaf(al3, po[k].w, v.w);
        xg[FI(k)] = v;
        const float4 q = qv[k];
        if (!dn0) r[k].x = fmaf(-al0, q.x, r[k].x);
        if (!dn1) r[k].y = fmaf(-al1, q.y, r[k].y);
        if (!dn2) r[k].z = fmaf(-al2, q.z, r[k].z);
        if (!dn3) r[k].w = fmaf(-al3, q.w, r[k].w);
        dot4(part, r[k], r[k]);
        const float dd = om * d0[k];
        put(cl, sm, L0, zo, rank, o0, fy0 + k, fx, make_float4(dd * r[k].x, dd * r[k].y, dd * r[k].z, dd * r[k].w));
      }
    }
    cluster_reduce<0>(cl, S, RK_RR, part, a, rank);
  }

  // ---- the solution into the output block
  const float4* xg = XG;
#pragma unroll
  for (int k = 0; k < FINE_ITEMS; ++k) {
    if (k >= fn) break;
    const int i = FI(k);
    const float4 v = xg[i];
    const size_t node = (size_t)o0.r0 * nx0 + i;
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (col0 + u < w) dst[node * ldd + col0 + u] = (TD)comp(v, u);
  }
#undef XG
#undef QG
#undef FI
  if (rank == 0 && threadIdx.x < 4 && a.iters && col0 + (int)threadIdx.x < w)
    a.iters[col0 + threadIdx.x] = S.cs[threadIdx.x].iters;
  // no CTA leaves while another may still read its shared memory
  cluster_sync_all();
}


// The finest-grid sweep of the wide solver: its nodes one at a time, the 9
// neighbours loaded per node (L1 serves the re-reads); a rolling window as in
// fine_sweep would hold 9 more float4 registers across the nodes, which the
// 64-register budget of two CTAs per SM cannot spare.
template <typename F>
__device__ __forceinline__ void wide_sweep(const float* __restrict__ ST, const float4* X, int W, int nx, int fy0,
                                           int fx, int fn, F f) {
#pragma unroll
  for (int k = 0; k < FINE_ITEMS; ++k) {
    if (k >= fn) break;
    const int c = (fy0 + k + 1) * W + fx + 1;
    const float4 ax = apply9(ST + ((fy0 + k) * nx + fx) * 9, X, W, c);
    f(k, c, ax, X[c]);
  }
}

// Global working set of the wide solver, per cluster: the finest grid's iterate
// and its partner as padded float4 grids [(ny + 2) x (nx + 2)] (zero border,
// never written), and r, p, x, A p as float4 per node.
struct WideArgs {
  float4* zs;       // [cluster][2][(ny+2)(nx+2)]
  float4* vecs;     // [cluster][4][n]: r, p, x, q
};

// The solver for batches wider than one wave of k_inner_cluster: the same
// method and the same coarse-grid code, with the finest grid in global memory
// (L2-resident at the sizes the plan admits) instead of shared memory, so a CTA
// needs only the coarse grids on chip (two CTAs per SM, 64 registers each) and
// all clusters of a 126-column batch are resident at once. Each CTA computes
// its strip of the finest grid reading its neighbours' rows directly; the
// cluster barrier (release/acquire at cluster scope) orders those accesses. r,
// p, x and A p live per node in the cluster's vectors; the strip's nodes stay
// with their thread as in k_inner_cluster.
template <typename TS, typename TD>
__global__ void __launch_bounds__(CNT, 2)
    k_inner_cluster_wide(const CPlan P, const TS* __restrict__ src, int lds, TD* __restrict__ dst, int ldd, int w,
                         const CArgs a, const WideArgs wa) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ CLevel L[CMAXG];
  __shared__ CShared S;
  const cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int cid = (int)(blockIdx.x / CLN);
  const int col0 = cid * 4;
  const int G = P.G, gs = P.gs, nu = a.nu;
  const float om = a.om;

  // ---- set-up of the coarse grids (as in k_inner_cluster, level 0 excluded)
#pragma unroll
  for (int g = 0; g < CMAXG; ++g)
    if ((int)threadIdx.x == g) L[g] = P.L[g];
  if (threadIdx.x < 4) {
    S.cs[threadIdx.x] = ColState{0.0, 0.0, 0, 1};
    S.alpha[threadIdx.x] = 0.f;
    S.beta[threadIdx.x] = 0.f;
  }
  __syncthreads();
  for (int g = 1; g < G; ++g) {
    const CLevel& l = L[g];
    const Own o = own_rows(l, rank);
    if (o.nr == 0) continue;
    stage_floats(sp<float>(sm, l.st), l.gst + (size_t)o.r0 * l.nx * 9, o.nr * l.nx * 9);
  }
  for (int g = 1; g < G; ++g) {
    const CLevel& l = L[g];
    const unsigned end = g + 1 < G ? L[g + 1].b : P.bytes;
    float4* z = reinterpret_cast<float4*>(sm);
    for (int i = (int)(l.b / 16) + threadIdx.x; i < (int)(l.st / 16); i += CNT) z[i] = f4(0.f);
    for (int i = (int)(l.di / 16) + threadIdx.x; i < (int)(end / 16); i += CNT) z[i] = f4(0.f);
  }
  __syncthreads();
  for (int g = 1; g < G; ++g) {
    const CLevel& l = L[g];
    const Own o = own_rows(l, rank);
    if (o.nr == 0) continue;
    float* di = sp<float>(sm, l.di);
    const int lo = max(o.r0 - 1, 0) - o.r0, hi = min(o.r0 + o.nr + 1, l.ny) - o.r0;
    for (int i = threadIdx.x; i < (hi - lo) * l.nx; i += CNT) {
      const int ly = lo + i / l.nx, x = i % l.nx;
      copy_async4(di + pidx(l, ly, x), l.gdi + (size_t)(o.r0 + ly) * l.nx + x);
    }
  }

  // ---- finest grid in global memory: this CTA's strip as local rows (row 0 =
  // grid row r0); thread nodes as in k_inner_cluster
  const CLevel& L0 = L[0];
  const Own o0 = own_rows(L0, rank);
  const int nx0 = L0.nx, W0 = nx0 + 2;
  const size_t padn = (size_t)(L0.ny + 2) * W0, n0 = (size_t)L0.nx * L0.ny;
  float4* const bufA = wa.zs + (size_t)cid * 2 * padn + (size_t)o0.r0 * W0;
  float4* const bufB = bufA + padn;
  float4* const GR = wa.vecs + (size_t)cid * 4 * n0 + (size_t)o0.r0 * nx0;
  float4* const GP = GR + n0;
  float4* const GX = GP + n0;
  float4* const GQ = GX + n0;
  const float* ST0 = L0.gst + (size_t)o0.r0 * nx0 * 9;
  const float* DI0 = L0.gdi + (size_t)o0.r0 * nx0;
  const int fx = threadIdx.x % nx0, fy0 = P.fine_h * ((int)threadIdx.x / nx0);
  const int fn = (int)threadIdx.x < (CNT / nx0) * nx0 ? max(0, min(P.fine_h, o0.nr - fy0)) : 0;
#define FI(k) ((fy0 + (k)) * nx0 + fx)
#define FC(k) ((fy0 + (k) + 1) * W0 + fx + 1)
  float4* Z = bufA;
  float4* Sb = bufB;
  float4 part = f4(0.f);
#pragma unroll
  for (int k = 0; k < FINE_ITEMS; ++k) {
    if (k < fn) {
      const int i = FI(k);
      const size_t node = (size_t)o0.r0 * nx0 + i;
      float v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = col0 + u < w ? (float)src[node * lds + col0 + u] : 0.f;
      const float4 r = make_float4(v[0], v[1], v[2], v[3]);
      GR[i] = r;
      GP[i] = f4(0.f);
      GX[i] = f4(0.f);
      dot4(part, r, r);
      const float dd = om * DI0[i];
      Z[FC(k)] = make_float4(dd * v[0], dd * v[1], dd * v[2], dd * v[3]);
    }
  }
  copy_async_wait();
  cluster_reduce<CLN>(cl, S, RK_INIT, part, a, rank);

  const int cap = (a.fixed > 0 ? a.fixed : a.maxit) + 1;
  for (int it = 0; it < cap && S.active; ++it) {
    // ---- finest grid down: sweeps 2..nu, residual, restriction
    for (int s = 1; s < nu; ++s) {
      wide_sweep(ST0, Z, W0, nx0, fy0, fx, fn, [&](int k, int c, const float4& ax, const float4& xc) {
        const float4 r = GR[FI(k)];
        const float dd = om * DI0[FI(k)];
        Sb[c] = make_float4(fmaf(dd, r.x - ax.x, xc.x), fmaf(dd, r.y - ax.y, xc.y), fmaf(dd, r.z - ax.z, xc.z),
                            fmaf(dd, r.w - ax.w, xc.w));
      });
      cluster_sync_all();
      float4* t = Z; Z = Sb; Sb = t;
    }
    wide_sweep(ST0, Z, W0, nx0, fy0, fx, fn, [&](int k, int c, const float4& ax, const float4&) {
      Sb[c] = sub4(GR[FI(k)], ax);
    });
    cluster_sync_all();
    restrict_rows(cl, sm, L0, o0, Sb, L[1], rank);
    cluster_sync_all();
    // ---- coarse grids
    for (int g = 1; g < gs; ++g) level_down(cl, sm, L, g, rank, nu, om);
    if (rank == 0) block_levels(cl, sm, L, gs, G, nu, om);
    cluster_sync_all();
    for (int g = gs - 1; g >= 1; --g) level_up(cl, sm, L, g, G, rank, nu, om);
    // ---- finest grid up; the last sweep also sums r . z
    const float4* XC = sp<float4>(sm, final_buf(L[1], G == 2, nu));
    const int Wc = L[1].nx + 2;
    for (int s = 1; s <= nu; ++s) {
      part = f4(0.f);
      wide_sweep(ST0, Z, W0, nx0, fy0, fx, fn, [&](int k, int c, const float4& ax, const float4& xc) {
        const float4 r = GR[FI(k)];
        const float dd = om * DI0[FI(k)];
        float4 v;
        if (s == 1) {
          const int y = o0.r0 + fy0 + k;
          float4 apc, pc;
          coarse_corr(ST0 + FI(k) * 9, XC, Wc, patch_centre(L[1], rank, y, fx), y & 1, fx & 1, apc, pc);
          const float4 xv = add4(xc, pc);
          v = make_float4(fmaf(dd, r.x - (ax.x + apc.x), xv.x), fmaf(dd, r.y - (ax.y + apc.y), xv.y),
                          fmaf(dd, r.z - (ax.z + apc.z), xv.z), fmaf(dd, r.w - (ax.w + apc.w), xv.w));
        } else {
          v = make_float4(fmaf(dd, r.x - ax.x, xc.x), fmaf(dd, r.y - ax.y, xc.y), fmaf(dd, r.z - ax.z, xc.z),
                          fmaf(dd, r.w - ax.w, xc.w));
        }
        Sb[c] = v;
        dot4(part, r, v);
      });
      if (s == nu) cluster_reduce<CLN>(cl, S, RK_RHO, part, a, rank);
      else cluster_sync_all();
      float4* t = Z; Z = Sb; Sb = t;
    }
    // ---- p = z + beta p, q = A z + beta q_old, p . q
    {
      const float4 bt = make_float4(S.beta[0], S.beta[1], S.beta[2], S.beta[3]);
      part = f4(0.f);
      wide_sweep(ST0, Z, W0, nx0, fy0, fx, fn, [&](int k, int, const float4& az, const float4& z) {
        const int i = FI(k);
        const float4 po = GP[i];
        const float4 qo = it > 0 ? GQ[i] : f4(0.f);
        const float4 p = make_float4(fmaf(bt.x, po.x, z.x), fmaf(bt.y, po.y, z.y), fmaf(bt.z, po.z, z.z),
                                     fmaf(bt.w, po.w, z.w));
        const float4 q = make_float4(fmaf(bt.x, qo.x, az.x), fmaf(bt.y, qo.y, az.y), fmaf(bt.z, qo.z, az.z),
                                     fmaf(bt.w, qo.w, az.w));
        GP[i] = p;
        GQ[i] = q;
        dot4(part, p, q);
      });
    }
    cluster_reduce<CLN>(cl, S, RK_PQ, part, a, rank);
    // ---- x += alpha p, r -= alpha q on the unfinished columns; r . r; the
    // next V-cycle's first sweep om D^-1 r
    {
      const float al0 = S.alpha[0], al1 = S.alpha[1], al2 = S.alpha[2], al3 = S.alpha[3];
      const bool dn0 = S.cs[0].done, dn1 = S.cs[1].done, dn2 = S.cs[2].done, dn3 = S.cs[3].done;
      const bool up0 = !dn0 && col0 < w, up1 = !dn1 && col0 + 1 < w, up2 = !dn2 && col0 + 2 < w,
                 up3 = !dn3 && col0 + 3 < w;
      part = f4(0.f);
#pragma unroll
      for (int k = 0; k < FINE_ITEMS; ++k) {
        if (k >= fn) break;
        const int i = FI(k);
        const float4 p = GP[i], q = GQ[i];
        float4 x = GX[i], r = GR[i];
        if (up0) x.x = fmaf(al0, p.x, x.x);
        if (up1) x.y = fmaf(al1, p.y, x.y);
        if (up2) x.z = fmaf(al2, p.z, x.z);
        if (up3) x.w = fmaf(al3, p.w, x.w);
        if (!dn0) r.x = fmaf(-al0, q.x, r.x);
        if (!dn1) r.y = fmaf(-al1, q.y, r.y);
        if (!dn2) r.z = fmaf(-al2, q.z, r.z);
        if (!dn3) r.w = fmaf(-al3, q.w, r.w);
        GX[i] = x;
        GR[i] = r;
        dot4(part, r, r);
        const float dd = om * DI0[i];
        Z[FC(k)] = make_float4(dd * r.x, dd * r.y, dd * r.z, dd * r.w);
      }
    }
    cluster_reduce<CLN>(cl, S, RK_RR, part, a, rank);
  }

  // ---- the solution into the output block
#pragma unroll
  for (int k = 0; k < FINE_ITEMS; ++k) {
    if (k >= fn) break;
    const int i = FI(k);
    const float4 v = GX[i];
    const size_t node = (size_t)o0.r0 * nx0 + i;
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (col0 + u < w) dst[node * ldd + col0 + u] = (TD)comp(v, u);
  }
#undef FI
#undef FC
  if (rank == 0 && threadIdx.x < 4 && a.iters && col0 + (int)threadIdx.x < w)
    a.iters[col0 + threadIdx.x] = S.cs[threadIdx.x].iters;
  cluster_sync_all();
}

}  // namespace

// ------------------------------------------------------------ host side ---

// Host-side state of the cluster solvers (h->cl_plan).
struct ClusterSolver {
  CPlan P{};                  // k_inner_cluster, clusters of 8: the whole hierarchy on chip
  CPlan P16{};                // k_inner_cluster, clusters of 16 (half the rows per CTA)
  CPlan Pw{};                 // k_inner_cluster_wide: the coarse grids on chip
  int maxcl = 0, maxcl16 = 0, maxclw = 0;   // clusters resident at once
  int xcap = 0;               // clusters the x / A p scratch holds
  float4* xs = nullptr;       // k_inner_cluster: x and A p per cluster
  float4* wzs = nullptr;      // k_inner_cluster_wide: padded finest-grid iterates
  float4* wvecs = nullptr;    // k_inner_cluster_wide: r, p, x, A p
};

// Raise kern's dynamic shared-memory limit to at least `bytes`. The limit
// belongs to the function, not to a problem: it is never lowered, so the plan
// of one problem does not invalidate the launches of another.
template <typename K>
static bool allow_smem(K kern, unsigned bytes) {
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return false;
  if (fa.maxDynamicSharedSizeBytes >= (int)bytes) return true;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
}

// Clusters of `cln` CTAs of kernel kern resident at once with `bytes` of
// dynamic shared memory (0 if it cannot run). Clusters of more than 8 CTAs
// are a non-portable size the kernel has to opt in to.
template <typename K>
static int max_clusters(K kern, unsigned bytes, int optin, int cln) {
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return 0;
  if ((long long)bytes + (long long)fa.sharedSizeBytes > optin) return 0;
  if (!allow_smem(kern, bytes)) return 0;
  if (cln > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cln);
  cfg.blockDim = dim3(CNT);
  cfg.dynamicSmemBytes = bytes;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cln;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess) return 0;
  return nclusters;
}

// The shared-memory plan of the hierarchy for clusters of `cln` CTAs: grids
// with at least cln rows in row strips of ceil(ny / cln) rows, the smaller
// ones on CTA 0 alone; with `wide` the finest grid takes no shared memory.
// False when the hierarchy does not fit the scheme (the caller then leaves
// that solver out).
static bool build_plan(const sg_problem* h, int cln, bool wide, CPlan& P) {
  const int G = (int)h->grids.size();
  if (G < 2 || G > CMAXG) return false;
  P = CPlan{};
  unsigned off = 0;
  auto take = [&](size_t bytes) {
    const unsigned r = off;
    off += (unsigned)((bytes + 15) & ~(size_t)15);
    return r;
  };
  int gs = G;
  for (int g = 0; g < G; ++g) {
    const GridLevel& gr = h->grids[g];
    CLevel& l = P.L[g];
    if (gr.nx != gr.ny || !gr.st32 || !gr.dinv32) return false;
    l.nx = gr.nx;
    l.ny = gr.ny;
    l.single = gr.ny < cln;
    l.rows = l.single ? gr.ny : (gr.ny + cln - 1) / cln;
    if (l.single) {
      if (gs == G) gs = g;
    } else if (gs < G) {
      return false;   // strips below a grid held by CTA 0
    }
    const size_t vec = (size_t)(l.rows + 2) * (l.nx + 2) * 16;
    const size_t stb = (size_t)l.rows * l.nx * 9 * sizeof(float);
    const size_t dib = (size_t)(l.rows + 2) * (l.nx + 2) * sizeof(float);
    l.gst = gr.st32;
    l.gdi = gr.dinv32;
    if (g == 0 && wide) continue;   // the finest grid lives in global memory
    l.b = g > 0 ? take(vec) : 0;
    l.x = take(vec);
    l.y = take(vec);
    l.st = take(stb);
    l.di = g > 0 ? take(dib) : 0;
  }
  if (gs == 0 || gs == G) return false;
  if (P.L[0].nx > CNT) return false;
  P.fine_h = (P.L[0].rows + CNT / P.L[0].nx - 1) / (CNT / P.L[0].nx);   // finest-grid rows per thread
  if (P.fine_h > FINE_ITEMS) return false;
  for (int g = 0; g + 1 < gs; ++g)   // strips of consecutive grids line up (row 2Y+1 over row Y)
    if (P.L[g].rows != 2 * P.L[g + 1].rows || P.L[g + 1].nx != (P.L[g].nx - 1) / 2) return false;
  P.G = G;
  P.gs = gs;
  P.bytes = off;
  return true;
}

// Build the shared-memory plans of the hierarchy and decide which cluster
// solvers can run it (h->cl_plan stays null when none can). Any CUDA error
// on this path only disables the cluster solvers; it is cleared.
int cluster_setup(sg_problem* h) {
  const char* ev = getenv("SGHSC_NO_CLUSTER");
  if (ev && ev[0] == '1') return SG_OK;
  const char* ev16 = getenv("SGHSC_NO_CLUSTER16");
  CPlan P{}, P16{}, Pw{};
  if (!build_plan(h, CLN, false, P) || !build_plan(h, CLN, true, Pw)) return SG_OK;
  const bool try16 = !(ev16 && ev16[0] == '1') && build_plan(h, 2 * CLN, false, P16);
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device) != cudaSuccess) {
    cudaGetLastError();
    return SG_OK;
  }
  auto min4 = [](int a, int b, int c, int d) { return std::min(std::min(a, b), std::min(c, d)); };
  auto onchip = [&](const CPlan& Q, int cln) {
    return min4(max_clusters(k_inner_cluster<double, float>, Q.bytes, optin, cln),
                max_clusters(k_inner_cluster<float, float>, Q.bytes, optin, cln),
                max_clusters(k_inner_cluster<double, double>, Q.bytes, optin, cln),
                max_clusters(k_inner_cluster<float, double>, Q.bytes, optin, cln));
  };
  const int maxcl = onchip(P, CLN);
  const int maxcl16 = try16 ? onchip(P16, 2 * CLN) : 0;
  const int maxclw = min4(max_clusters(k_inner_cluster_wide<double, float>, Pw.bytes, optin, CLN),
                          max_clusters(k_inner_cluster_wide<float, float>, Pw.bytes, optin, CLN),
                          max_clusters(k_inner_cluster_wide<double, double>, Pw.bytes, optin, CLN),
                          max_clusters(k_inner_cluster_wide<float, double>, Pw.bytes, optin, CLN));
  cudaGetLastError();
  if (maxcl < 1 && maxclw < 1 && maxcl16 < 1) return SG_OK;
  ClusterSolver* cs = new ClusterSolver();
  cs->P = P;
  cs->P16 = P16;
  cs->Pw = Pw;
  cs->maxcl = std::max(maxcl, 0);
  cs->maxcl16 = std::max(maxcl16, 0);
  cs->maxclw = std::max(maxclw, 0);
  cs->P.maxcl = cs->maxcl;
  cs->P16.maxcl = cs->maxcl16;
  cs->Pw.maxcl = cs->maxclw;
  cs->xcap = std::max(cs->maxcl, cs->maxcl16);
  h->cl_plan = cs;   // owned from here on (cluster_free)
  const size_t n = (size_t)P.L[0].nx * P.L[0].ny, padn = (size_t)(P.L[0].ny + 2) * (P.L[0].nx + 2);
  if (cs->xcap > 0) SG_TRY_CUDA(cudaMalloc((void**)&cs->xs, 2 * (size_t)cs->xcap * n * sizeof(float4)));
  if (cs->maxclw > 0) {
    SG_TRY_CUDA(cudaMalloc((void**)&cs->wzs, 2 * (size_t)cs->maxclw * padn * sizeof(float4)));
    SG_TRY_CUDA(cudaMemset(cs->wzs, 0, 2 * (size_t)cs->maxclw * padn * sizeof(float4)));   // zero borders
    SG_TRY_CUDA(cudaMalloc((void**)&cs->wvecs, 4 * (size_t)cs->maxclw * n * sizeof(float4)));
  }
  return SG_OK;
}

void cluster_free(sg_problem* h) {
  ClusterSolver* cs = (ClusterSolver*)h->cl_plan;
  if (!cs) return;
  cudaFree(cs->xs);
  cudaFree(cs->wzs);
  cudaFree(cs->wvecs);
  delete cs;
  h->cl_plan = nullptr;
}

// Which cluster solver an FP32 batch of w columns takes: 3 = the on-chip one
// with clusters of 16 CTAs when all of them are resident at once (half the
// rows per CTA: the phases of the latency-bound solve are shorter), 1 = the
// on-chip one with clusters of 8 when all of them are (a second wave would
// double the solve), 2 = the wide one (finest grid in global memory) when its
// clusters are, 0 = none of them (the stand-alone kernels).
// The autotuner's choice for the width (sg_autotune) takes precedence when
// it is one of the eligible solvers.
static bool path_eligible(const ClusterSolver* cs, int w, int path) {
  const int ncl = ceil_div(w, 4);
  if (path == 3) return ncl <= cs->maxcl16;
  if (path == 1) return ncl <= cs->maxcl;
  if (path == 2) return ncl <= cs->maxclw;
  return path == 0;
}

static int cluster_path(const sg_problem* h, int dtype, int w) {
  const ClusterSolver* cs = (const ClusterSolver*)h->cl_plan;
  if (dtype != SG_F32 || !cs) return 0;
  const auto it = h->inner_pick.find(w);
  if (it != h->inner_pick.end() && path_eligible(cs, w, it->second)) return it->second;
  for (int path : {3, 1, 2})
    if (path_eligible(cs, w, path)) return path;
  return 0;
}

std::vector<int> inner_path_candidates(const sg_problem* h, int w) {
  std::vector<int> c{0};
  const ClusterSolver* cs = (const ClusterSolver*)h->cl_plan;
  if (!cs) return c;
  for (int path : {3, 1, 2})
    if (path_eligible(cs, w, path)) c.push_back(path);
  return c;
}

bool cluster_usable(const sg_problem* h, int dtype, int w) { return cluster_path(h, dtype, w) != 0; }

}  // namespace sghsc

extern "C" int sg_inner_cluster(const sg_problem* h) { return h && h->cl_plan ? 1 : 0; }

extern "C" int sg_inner_path(const sg_problem* h, int w, int dtype) {
  if (!h || w <= 0) return 0;
  return sghsc::cluster_path(h, dtype, w);
}

namespace sghsc {

int inner_solve_cluster(sg_problem* h, const void* src, int lds, int src_t, void* dst, int ldd, int dst_t, int w,
                        const sg_prec_opts& o, cudaStream_t s) {
  const ClusterSolver& cs = *(const ClusterSolver*)h->cl_plan;
  const int path = cluster_path(h, SG_F32, w);
  const CPlan& P = path == 2 ? cs.Pw : path == 3 ? cs.P16 : cs.P;
  const int cln = path == 3 ? 2 * CLN : CLN;
  CArgs a;
  a.om = (float)o.omega;
  a.nu = o.nu;
  a.tol2 = o.inner_tol * o.inner_tol;
  a.maxit = o.inner_maxit;
  a.fixed = o.inner_fixed_iters;
  a.status = h->status;
  a.iacc = h->iacc;
  a.iters = h->iw32.iters && h->iw32.wcap >= w ? h->iw32.iters : nullptr;
  a.xs = cs.xs;
  a.qs = cs.xs ? cs.xs + (size_t)cs.xcap * P.L[0].nx * P.L[0].ny : nullptr;
  WideArgs wa;
  wa.zs = cs.wzs;
  wa.vecs = cs.wvecs;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(ceil_div(w, 4) * cln));
  cfg.blockDim = dim3(CNT);
  cfg.dynamicSmemBytes = P.bytes;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cln;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const bool s64 = src_t == SG_F64, d64 = dst_t == SG_F64;
  if (path == 2) {
    if (s64 && d64)
      SG_TRY_CUDA(cudaLaunchKernelEx(&cfg, k_inner_cluster_wide<double, double>, P, (const double*)src, lds, (double*)dst, ldd, w, a, wa));
    else if (s64)
      SG_TRY_CUDA(cudaLaunchKernelEx(&cfg, k_inner_cluster_wide<double, float>, P, (const double*)src, lds, (float*)dst, ldd, w, a, wa));
    else if (d64)
      SG_TRY_CUDA(cudaLaunchKernelEx(&cfg, k_inner_cluster_wide<float, double>, P, (const float*)src, lds, (double*)dst, ldd, w, a, wa));
    else
      SG_TRY_CUDA(cudaLaunchKernelEx(&cfg, k_inner_cluster_wide<float, float>, P, (const float*)src, lds, (float*)dst, ldd, w, a, wa));
  } else {
    if (s64 && d64)
      SG_TRY_CUDA(cudaLaunchKernelEx(&cfg, k_inner_cluster<double, double>, P, (const double*)src, lds, (double*)dst, ldd, w, a));
    else if (s64)
      SG_TRY_CUDA(cudaLaunchKernelEx(&cfg, k_inner_cluster<double, float>, P, (const double*)src, lds, (float*)dst, ldd, w, a));
    else if (d64)
      SG_TRY_CUDA(cudaLaunchKernelEx(&cfg, k_inner_cluster<float, double>, P, (const float*)src, lds, (double*)dst, ldd, w, a));
    else
      SG_TRY_CUDA(cudaLaunchKernelEx(&cfg, k_inner_cluster<float, float>, P, (const float*)src, lds, (float*)dst, ldd, w, a));
  }
  note_launch();
  return SG_OK;
}

}  // namespace sghsc
