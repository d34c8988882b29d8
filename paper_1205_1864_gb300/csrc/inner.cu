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
// Thread mapping: a block has k*w threads (k = max(1, 256 / w)), thread t
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
//   k_vcycle_coarse   all grids with <= 1024 nodes: one block per 4 columns
//                     runs the rest of the V-cycle in shared memory.
#include <algorithm>

#include "graph.cuh"
#include "sghsc_internal.cuh"

namespace sghsc {

constexpr int CB_MAX_NODES = 1024;
constexpr int CPB = 4;
constexpr int MAX_LEVELS = 16;

struct Shape {
  int w, k, bdim, grid;
};

static Shape make_shape(const sg_problem* h, int nodes, int w) {
  Shape s;
  s.w = w;
  s.k = w <= 256 ? std::max(1, 256 / w) : 1;
  s.bdim = s.k * w;
  s.grid = std::max(1, std::min(ceil_div(nodes, s.k), h->num_sms * 8));
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
  double* part;
  int ldp;
  InnerCtl* ctl;
  double *rho, *pq, *rr, *bb, *alpha, *beta;
  int *done, *iters;
  int* status;
  double tol2;
  int maxit, fixed;
  cudaGraphConditionalHandle cond;
  int has_cond;
};

__device__ __forceinline__ void thread_pos(int w, int k, int& col, int& node0, int& nstep) {
  col = threadIdx.x % w;
  node0 = blockIdx.x * k + threadIdx.x / w;
  nstep = gridDim.x * k;
}

// Per-column block partial: the k threads of column c sum in a fixed order.
__device__ __forceinline__ void block_col_reduce(double v, int w, int k, double* part, int ldp) {
  __shared__ double red[1024];
  red[threadIdx.x] = v;
  __syncthreads();
  if ((int)threadIdx.x < w) {
    double s = 0.0;
    for (int m = 0; m < k; ++m) s += red[threadIdx.x + m * w];
    part[(size_t)blockIdx.x * ldp + threadIdx.x] = s;
  }
}

// True in the last block to finish (threadFenceReduction pattern).
__device__ __forceinline__ bool last_block(unsigned* ticket) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Column-wise CG scalar updates from the block partials (last block only).
__device__ void fin_columns(const FinArgs& f, int op, int w, int nblk) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  const int c = threadIdx.x;
  if (c < w) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += __ldcg(&f.part[(size_t)b * f.ldp + c]);
    if (op == FIN_INIT) {
      f.bb[c] = s;
      f.done[c] = !(s > 0.0);
      f.iters[c] = 0;
      f.beta[c] = 0.0;
    } else if (!f.done[c]) {
      if (op == FIN_RHO) {
        f.beta[c] = f.iters[c] == 0 ? 0.0 : s / f.rho[c];
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
      }
    }
    if (!f.done[c]) atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (op == FIN_INIT) f.ctl->it = 0;
    if (op == FIN_CONV) f.ctl->it += 1;
    f.ctl->active = cnt;
    if ((op == FIN_INIT || op == FIN_CONV) && f.has_cond) cudaGraphSetConditional(f.cond, cnt > 0 ? 1u : 0u);
    f.ctl->ticket = 0;
  }
}

__device__ __forceinline__ void reduce_finalize(const FinArgs& f, double v, int w, int k, int op) {
  block_col_reduce(v, w, k, f.part, f.ldp);
  if (last_block(&f.ctl->ticket)) fin_columns(f, op, w, gridDim.x);
}

// sum_j a_ij v_j over the 9-point stencil of node (x, y) (v node-major, ld w)
template <typename T>
__device__ __forceinline__ T stencil_dot(const T* __restrict__ s9, int nx, int ny, int x, int y,
                                         const T* __restrict__ v, int w, int col) {
  T acc = T(0);
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
    const int yy = y + dy;
    if (yy < 0 || yy >= ny) continue;
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const int xx = x + dx;
      if (xx < 0 || xx >= nx) continue;
      acc += s9[(dy + 1) * 3 + (dx + 1)] * v[(size_t)(yy * nx + xx) * w + col];
    }
  }
  return acc;
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

// ---------------------------------------------------------------- V-cycle ---

// one sweep from zero: x = omega D^{-1} b
template <typename T>
__global__ void k_smooth0(int n, int w, int k, const T* __restrict__ dinv, const T* __restrict__ b,
                          T* __restrict__ x, T om, const int* __restrict__ done) {
  int col, node, nstep;
  thread_pos(w, k, col, node, nstep);
  if (done[col]) return;
  for (; node < n; node += nstep) {
    const size_t i = (size_t)node * w + col;
    x[i] = om * dinv[node] * b[i];
  }
}

// two sweeps from zero: x1 = omega D^{-1} b, x2 = x1 + omega D^{-1} (b - A x1)
template <typename T>
__global__ void k_smooth00(int nx, int ny, int w, int k, const T* __restrict__ st, const T* __restrict__ dinv,
                           const T* __restrict__ b, T* __restrict__ x, T om, const int* __restrict__ done) {
  int col, node, nstep;
  thread_pos(w, k, col, node, nstep);
  if (done[col]) return;
  const int n = nx * ny;
  for (; node < n; node += nstep) {
    const int y = node / nx, xx0 = node - y * nx;
    const T* s9 = st + (size_t)node * 9;
    T ax1 = T(0);
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int yy = y + dy;
      if (yy < 0 || yy >= ny) continue;
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int xx = xx0 + dx;
        if (xx < 0 || xx >= nx) continue;
        const int j = yy * nx + xx;
        ax1 += s9[(dy + 1) * 3 + (dx + 1)] * (om * dinv[j] * b[(size_t)j * w + col]);
      }
    }
    const size_t i = (size_t)node * w + col;
    const T bi = b[i], di = dinv[node];
    const T x1 = om * di * bi;
    x[i] = x1 + om * di * (bi - ax1);
  }
}

// xo = xi + omega D^{-1} (b - A xi); with DOT also the partials of b . xo and FIN_RHO
template <typename T, bool DOT>
__global__ void k_jacobi(int nx, int ny, int w, int k, const T* __restrict__ st, const T* __restrict__ dinv,
                         const T* __restrict__ b, const T* __restrict__ xi, T* __restrict__ xo, T om, FinArgs f) {
  int col, node, nstep;
  thread_pos(w, k, col, node, nstep);
  typename Acc<T>::type acc = 0;
  if (!f.done[col]) {
    const int n = nx * ny;
    for (; node < n; node += nstep) {
      const int y = node / nx, x = node - y * nx;
      const size_t i = (size_t)node * w + col;
      const T bi = b[i];
      const T v = xi[i] + om * dinv[node] * (bi - stencil_dot(st + (size_t)node * 9, nx, ny, x, y, xi, w, col));
      xo[i] = v;
      if (DOT) acc += bi * v;
    }
  }
  if (DOT) reduce_finalize(f, (double)acc, w, k, FIN_RHO);
}

// bc = P^T (b - A x): coarse node (X, Y) gathers the 3x3 fine residuals around (2X+1, 2Y+1)
template <typename T>
__global__ void k_resid_restrict(int nxf, int nyf, int nxc, int nyc, int w, int k, const T* __restrict__ st,
                                 const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ bc,
                                 const int* __restrict__ done) {
  int col, node, nstep;
  thread_pos(w, k, col, node, nstep);
  if (done[col]) return;
  const int n = nxc * nyc;
  for (; node < n; node += nstep) {
    const int Y = node / nxc, X = node - Y * nxc;
    const int cx = 2 * X + 1, cy = 2 * Y + 1;
    T acc = T(0);
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const T wy = dy == 0 ? T(1) : T(0.5);
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const T wx = dx == 0 ? T(1) : T(0.5);
        const int fx = cx + dx, fy = cy + dy;
        const int f = fy * nxf + fx;
        const T r = b[(size_t)f * w + col] - stencil_dot(st + (size_t)f * 9, nxf, nyf, fx, fy, x, w, col);
        acc += wx * wy * r;
      }
    }
    bc[(size_t)node * w + col] = acc;
  }
}

// x' = x + P xc (on the fly), xo = x' + omega D^{-1} (b - A x'); DOT as k_jacobi
template <typename T, bool DOT>
__global__ void k_prolong_jacobi(int nxf, int nyf, int nxc, int nyc, int w, int k, const T* __restrict__ st,
                                 const T* __restrict__ dinv, const T* __restrict__ b, const T* __restrict__ x,
                                 const T* __restrict__ xc, T* __restrict__ xo, T om, FinArgs f) {
  int col, node, nstep;
  thread_pos(w, k, col, node, nstep);
  typename Acc<T>::type acc = 0;
  if (!f.done[col]) {
    const int n = nxf * nyf;
    for (; node < n; node += nstep) {
      const int y = node / nxf, x0 = node - y * nxf;
      const T* s9 = st + (size_t)node * 9;
      T ax = T(0);
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) {
        const int yy = y + dy;
        if (yy < 0 || yy >= nyf) continue;
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const int xx = x0 + dx;
          if (xx < 0 || xx >= nxf) continue;
          const int j = yy * nxf + xx;
          const T xj = x[(size_t)j * w + col] + prolong_at(xx, yy, nxc, nyc, xc, w, col);
          ax += s9[(dy + 1) * 3 + (dx + 1)] * xj;
        }
      }
      const size_t i = (size_t)node * w + col;
      const T xi = x[i] + prolong_at(x0, y, nxc, nyc, xc, w, col);
      const T bi = b[i];
      const T v = xi + om * dinv[node] * (bi - ax);
      xo[i] = v;
      if (DOT) acc += bi * v;
    }
  }
  if (DOT) reduce_finalize(f, (double)acc, w, k, FIN_RHO);
}

struct CoarseGrids {
  int g0, G;
  int nx[MAX_LEVELS], ny[MAX_LEVELS], off[MAX_LEVELS];
  const void* st[MAX_LEVELS];
  const void* dinv[MAX_LEVELS];
};

// The V-cycle from grid g0 down for CPB columns per block, entirely in shared
// memory: per grid a right-hand side, an iterate and a ping-pong buffer,
// [node][CPB]; stencils are read from global memory (shared by every block).
template <typename T>
__global__ void __launch_bounds__(256) k_vcycle_coarse(CoarseGrids L, int w, const T* __restrict__ bg,
                                                       T* __restrict__ xg, T om, int nu,
                                                       const int* __restrict__ done) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int c0 = blockIdx.x * CPB;
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  if ((int)threadIdx.x < CPB && c0 + (int)threadIdx.x < w && !done[c0 + threadIdx.x]) any = 1;
  __syncthreads();
  if (!any) return;
  auto B = [&](int g) { return sm + (size_t)3 * L.off[g] * CPB; };
  auto Xa = [&](int g) { return sm + (size_t)(3 * L.off[g] + L.nx[g] * L.ny[g]) * CPB; };
  auto Xb = [&](int g) { return sm + (size_t)(3 * L.off[g] + 2 * L.nx[g] * L.ny[g]) * CPB; };
  auto sdot = [&](const T* s9, int nx, int ny, int x, int y, const T* v, int cc) {
    T acc = T(0);
    for (int dy = -1; dy <= 1; ++dy) {
      const int yy = y + dy;
      if (yy < 0 || yy >= ny) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int xx = x + dx;
        if (xx < 0 || xx >= nx) continue;
        acc += s9[(dy + 1) * 3 + (dx + 1)] * v[(yy * nx + xx) * CPB + cc];
      }
    }
    return acc;
  };
  {
    const int n0 = L.nx[L.g0] * L.ny[L.g0];
    T* b0 = B(L.g0);
    for (int idx = threadIdx.x; idx < n0 * CPB; idx += blockDim.x) {
      const int node = idx / CPB, cc = idx - node * CPB, col = c0 + cc;
      b0[idx] = col < w ? bg[(size_t)node * w + col] : T(0);
    }
  }
  __syncthreads();
  T* cur[MAX_LEVELS];
  T* oth[MAX_LEVELS];
  for (int g = L.g0; g < L.G; ++g) {
    const int nx = L.nx[g], ny = L.ny[g], n = nx * ny;
    const T* st = (const T*)L.st[g];
    const T* dinv = (const T*)L.dinv[g];
    const T* b = B(g);
    T* c = Xa(g);
    T* o = Xb(g);
    if (g == L.G - 1) {  // coarsest grid (one node for square grids): exact solve
      for (int idx = threadIdx.x; idx < n * CPB; idx += blockDim.x) c[idx] = dinv[idx / CPB] * b[idx];
      __syncthreads();
      cur[g] = c;
      oth[g] = o;
      break;
    }
    for (int idx = threadIdx.x; idx < n * CPB; idx += blockDim.x) c[idx] = om * dinv[idx / CPB] * b[idx];
    __syncthreads();
    for (int s = 1; s < nu; ++s) {
      for (int idx = threadIdx.x; idx < n * CPB; idx += blockDim.x) {
        const int node = idx / CPB, cc = idx - node * CPB, y = node / nx, x = node - y * nx;
        o[idx] = c[idx] + om * dinv[node] * (b[idx] - sdot(st + node * 9, nx, ny, x, y, c, cc));
      }
      __syncthreads();
      T* t = c; c = o; o = t;
    }
    for (int idx = threadIdx.x; idx < n * CPB; idx += blockDim.x) {
      const int node = idx / CPB, cc = idx - node * CPB, y = node / nx, x = node - y * nx;
      o[idx] = b[idx] - sdot(st + node * 9, nx, ny, x, y, c, cc);
    }
    __syncthreads();
    const int nxc = L.nx[g + 1], nyc = L.ny[g + 1];
    T* bc = B(g + 1);
    for (int idx = threadIdx.x; idx < nxc * nyc * CPB; idx += blockDim.x) {
      const int node = idx / CPB, cc = idx - node * CPB, Y = node / nxc, X = node - Y * nxc;
      T acc = T(0);
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const T wgt = (dx == 0 ? T(1) : T(0.5)) * (dy == 0 ? T(1) : T(0.5));
          acc += wgt * o[((2 * Y + 1 + dy) * nx + (2 * X + 1 + dx)) * CPB + cc];
        }
      bc[idx] = acc;
    }
    __syncthreads();
    cur[g] = c;
    oth[g] = o;
  }
  for (int g = L.G - 2; g >= L.g0; --g) {
    const int nx = L.nx[g], ny = L.ny[g], n = nx * ny;
    const int nxc = L.nx[g + 1], nyc = L.ny[g + 1];
    const T* st = (const T*)L.st[g];
    const T* dinv = (const T*)L.dinv[g];
    const T* b = B(g);
    T* c = cur[g];
    T* o = oth[g];
    const T* xc = cur[g + 1];
    for (int idx = threadIdx.x; idx < n * CPB; idx += blockDim.x) {
      const int node = idx / CPB, cc = idx - node * CPB, y = node / nx, x = node - y * nx;
      c[idx] += prolong_at(x, y, nxc, nyc, xc + cc, CPB, 0);
    }
    __syncthreads();
    for (int s = 0; s < nu; ++s) {
      for (int idx = threadIdx.x; idx < n * CPB; idx += blockDim.x) {
        const int node = idx / CPB, cc = idx - node * CPB, y = node / nx, x = node - y * nx;
        o[idx] = c[idx] + om * dinv[node] * (b[idx] - sdot(st + node * 9, nx, ny, x, y, c, cc));
      }
      __syncthreads();
      T* t = c; c = o; o = t;
    }
    cur[g] = c;
  }
  const int n0 = L.nx[L.g0] * L.ny[L.g0];
  const T* x0 = cur[L.g0];
  for (int idx = threadIdx.x; idx < n0 * CPB; idx += blockDim.x) {
    const int node = idx / CPB, cc = idx - node * CPB, col = c0 + cc;
    if (col < w) xg[(size_t)node * w + col] = x0[idx];
  }
}

// ------------------------------------------------------------- batched CG ---

// r = src (cast), x = 0, ||b||^2 -> FIN_INIT (sets the loop condition)
template <typename TS, typename T>
__global__ void k_gather(int n, int w, int k, const TS* __restrict__ src, int lds, T* __restrict__ r,
                         T* __restrict__ x, FinArgs f) {
  int col, node, nstep;
  thread_pos(w, k, col, node, nstep);
  typename Acc<T>::type acc = 0;
  for (; node < n; node += nstep) {
    const size_t i = (size_t)node * w + col;
    const T v = (T)src[(size_t)node * lds + col];
    r[i] = v;
    x[i] = T(0);
    acc += v * v;
  }
  reduce_finalize(f, (double)acc, w, k, FIN_INIT);
}

template <typename T, typename TD>
__global__ void k_scatter(int n, int w, int k, const T* __restrict__ x, TD* __restrict__ dst, int ldd) {
  int col, node, nstep;
  thread_pos(w, k, col, node, nstep);
  for (; node < n; node += nstep) dst[(size_t)node * ldd + col] = (TD)x[(size_t)node * w + col];
}

// a . b per column -> op (used when the finest grid is inside the coarse block)
template <typename T>
__global__ void k_dot_fin(int n, int w, int k, const T* __restrict__ a, const T* __restrict__ b, FinArgs f, int op) {
  int col, node, nstep;
  thread_pos(w, k, col, node, nstep);
  typename Acc<T>::type acc = 0;
  if (!f.done[col])
    for (; node < n; node += nstep) {
      const size_t i = (size_t)node * w + col;
      acc += a[i] * b[i];
    }
  reduce_finalize(f, (double)acc, w, k, op);
}

// p_new = z + beta p_old (p_new = z on a column's first iteration), formed on the
// fly at the 9 neighbours; q = A_0 p_new; p_new . q -> FIN_ALPHA.
template <typename T>
__global__ void k_matvec_p(int nx, int ny, int w, int k, const T* __restrict__ st, const T* __restrict__ z,
                           T* pA, T* pB, T* __restrict__ q, FinArgs f) {
  int col, node, nstep;
  thread_pos(w, k, col, node, nstep);
  const int par = f.ctl->it & 1;
  const T* __restrict__ pold = par ? pB : pA;
  T* __restrict__ pnew = par ? pA : pB;
  typename Acc<T>::type acc = 0;
  if (!f.done[col]) {
    const bool first = f.iters[col] == 0;
    const T bt = first ? T(0) : (T)f.beta[col];
    const int n = nx * ny;
    for (; node < n; node += nstep) {
      const int y = node / nx, x0 = node - y * nx;
      const T* s9 = st + (size_t)node * 9;
      T s = T(0);
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) {
        const int yy = y + dy;
        if (yy < 0 || yy >= ny) continue;
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const int xx = x0 + dx;
          if (xx < 0 || xx >= nx) continue;
          const size_t j = (size_t)(yy * nx + xx) * w + col;
          const T pj = first ? z[j] : z[j] + bt * pold[j];
          s += s9[(dy + 1) * 3 + (dx + 1)] * pj;
        }
      }
      const size_t i = (size_t)node * w + col;
      const T pi = first ? z[i] : z[i] + bt * pold[i];
      pnew[i] = pi;
      q[i] = s;
      acc += pi * s;
    }
  }
  reduce_finalize(f, (double)acc, w, k, FIN_ALPHA);
}

// x += alpha p_new; r -= alpha q; r . r -> FIN_CONV (sets the loop condition)
template <typename T>
__global__ void k_update_xr(int n, int w, int k, const T* pA, const T* pB, const T* __restrict__ q,
                            T* __restrict__ x, T* __restrict__ r, FinArgs f) {
  int col, node, nstep;
  thread_pos(w, k, col, node, nstep);
  const T* __restrict__ pnew = (f.ctl->it & 1) ? pA : pB;
  typename Acc<T>::type acc = 0;
  if (!f.done[col]) {
    const T a = (T)f.alpha[col];
    for (; node < n; node += nstep) {
      const size_t i = (size_t)node * w + col;
      x[i] += a * pnew[i];
      const T rv = r[i] - a * q[i];
      r[i] = rv;
      acc += rv * rv;
    }
  }
  reduce_finalize(f, (double)acc, w, k, FIN_CONV);
}

// Accumulate per-column iteration counts into the handle's running totals.
__global__ void k_iter_stats(int w, const int* iters, long long* acc) {
  __shared__ long long tot;
  __shared__ int mx;
  if (threadIdx.x == 0) { tot = 0; mx = 0; }
  __syncthreads();
  if ((int)threadIdx.x < w) {
    atomicAdd((unsigned long long*)&tot, (unsigned long long)iters[threadIdx.x]);
    atomicMax(&mx, iters[threadIdx.x]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    acc[0] += tot;
    if (mx > acc[1]) acc[1] = mx;
  }
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
                  iw.alpha, iw.beta, iw.done, iw.iters, iw.ctl};
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
  f.done = iw.done;
  f.iters = iw.iters;
  f.status = h->status;
  f.tol2 = o.inner_tol * o.inner_tol;
  f.maxit = o.inner_maxit;
  f.fixed = o.inner_fixed_iters;
  f.cond = 0;
  f.has_cond = 0;
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
  const size_t smem = (size_t)3 * tot * CPB * sizeof(T);
  SG_TRY_CUDA(cudaFuncSetAttribute(k_vcycle_coarse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  { k_vcycle_coarse<T><<<ceil_div(w, CPB), 256, smem, s>>>(L, w, b, x, (T)o.omega, o.nu, done); ::sghsc::note_launch(); }
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
      const Shape sh = make_shape(h, h->grids[g].n, w);
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
    { k_prolong_jacobi<T, true><<<sh.grid, sh.bdim, 0, s>>>(G.nx, G.ny, C.nx, C.ny, w, sh.k, st, dinv, b, cur, xc, oth, om, *fdot); ::sghsc::note_launch(); }
  } else {
    { k_prolong_jacobi<T, false><<<sh.grid, sh.bdim, 0, s>>>(G.nx, G.ny, C.nx, C.ny, w, sh.k, st, dinv, b, cur, xc, oth, om, fz); ::sghsc::note_launch(); }
  }
  std::swap(cur, oth);
  for (int it = 1; it < o.nu; ++it) {
    if (it == o.nu - 1 && fdot) {
      { k_jacobi<T, true><<<sh.grid, sh.bdim, 0, s>>>(G.nx, G.ny, w, sh.k, st, dinv, b, cur, oth, om, *fdot); ::sghsc::note_launch(); }
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
  const Shape sh = make_shape(h, G.n, w);
  T* x = (T*)iw.x;
  T* r = (T*)iw.r;
  T* q = (T*)iw.q;
  T* pA = (T*)iw.pA;
  T* pB = (T*)iw.pB;
  const T* st = sizeof(T) == 8 ? (const T*)G.st64 : (const T*)G.st32;
  FinArgs fa = make_fin(h, iw, o);
  auto pre = [&](cudaStream_t ps, cudaGraphConditionalHandle cond) -> int {
    FinArgs f = fa;
    f.cond = cond;
    f.has_cond = 1;
    if (src_t == SG_F64)
      { k_gather<double, T><<<sh.grid, sh.bdim, 0, ps>>>(G.n, w, sh.k, (const double*)src, ld_src, r, x, f); ::sghsc::note_launch(); }
    else
      { k_gather<float, T><<<sh.grid, sh.bdim, 0, ps>>>(G.n, w, sh.k, (const float*)src, ld_src, r, x, f); ::sghsc::note_launch(); }
    SG_CHECK_LAUNCH();
    return SG_OK;
  };
  auto body = [&](cudaStream_t bs, cudaGraphConditionalHandle cond) -> int {
    FinArgs f = fa;
    f.cond = cond;
    f.has_cond = 1;
    const T* z = nullptr;
    SG_TRY(vcycle<T>(h, iw, 0, r, (T*)iw.z, (T*)iw.zt, w, o, bs, &f, &z));
    { k_matvec_p<T><<<sh.grid, sh.bdim, 0, bs>>>(G.nx, G.ny, w, sh.k, st, z, pA, pB, q, f); ::sghsc::note_launch(); }
    { k_update_xr<T><<<sh.grid, sh.bdim, 0, bs>>>(G.n, w, sh.k, pA, pB, q, x, r, f); ::sghsc::note_launch(); }
    SG_CHECK_LAUNCH();
    return SG_OK;
  };
  SG_TRY(capture_while(h, s, pre, body));
  if (dst_t == SG_F64)
    { k_scatter<T, double><<<sh.grid, sh.bdim, 0, s>>>(G.n, w, sh.k, x, (double*)dst, ld_dst); ::sghsc::note_launch(); }
  else
    { k_scatter<T, float><<<sh.grid, sh.bdim, 0, s>>>(G.n, w, sh.k, x, (float*)dst, ld_dst); ::sghsc::note_launch(); }
  { k_iter_stats<<<1, ((w + 31) / 32) * 32, 0, s>>>(w, iw.iters, h->iacc); ::sghsc::note_launch(); }
  SG_CHECK_LAUNCH();
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

}  // namespace sghsc
