// Elementwise kernels: precision casts between strided blocks and the FP64
// vector updates and dot products of the outer flexible CG (Sec. 5-6).
// Each reduction kernel writes block partials; the last block to finish sums
// them in block order (so results do not depend on scheduling) and updates
// the CG scalars on the device.
#include <algorithm>

#include "sghsc_internal.cuh"
#include "vec.cuh"

namespace sghsc {

template <typename TS, typename TD>
__global__ void k_cast(const TS* __restrict__ src, int lds, TD* __restrict__ dst, int ldd, int rows, int cols) {
  const long long total = (long long)rows * cols;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / cols), c = (int)(i - (long long)r * cols);
    dst[(size_t)r * ldd + c] = widen<TD>(src[(size_t)r * lds + c]);
  }
}

// dst = src, n doubles; 16-byte pieces when both are 16-byte aligned. Either
// side may be page-locked host memory (mapped into the device's address
// space): the SMs then move the data over the host link themselves.
__global__ void __launch_bounds__(512) k_copy64(const double* __restrict__ src, double* __restrict__ dst,
                                                long long n, int vec) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (vec) {
    const long long n2 = n / 2;
    const double2* s2 = reinterpret_cast<const double2*>(src);
    double2* d2 = reinterpret_cast<double2*>(dst);
    for (long long i = t; i < n2; i += stride) d2[i] = s2[i];
    if (t == 0 && (n & 1)) dst[n - 1] = src[n - 1];
  } else {
    for (long long i = t; i < n; i += stride) dst[i] = src[i];
  }
}

int launch_copy64(const double* src, double* dst, long long n, int num_sms, cudaStream_t s) {
  if (n <= 0) return SG_OK;
  const int vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0;
  const int grid = (int)std::min<long long>((n / (vec ? 2 : 1) + 511) / 512, (long long)num_sms * 8);
  { k_copy64<<<std::max(grid, 1), 512, 0, s>>>(src, dst, n, vec); ::sghsc::note_launch(); }
  SG_CHECK_LAUNCH();
  return SG_OK;
}

int launch_cast(const void* src, int src_t, int lds, void* dst, int dst_t, int ldd, int rows, int cols,
                cudaStream_t s) {
  const long long total = (long long)rows * cols;
  if (total == 0) return SG_OK;
  const int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
  if (src_t == SG_F64 && dst_t == SG_F32)
    { k_cast<double, float><<<grid, 256, 0, s>>>((const double*)src, lds, (float*)dst, ldd, rows, cols); ::sghsc::note_launch(); }
  else if (src_t == SG_F32 && dst_t == SG_F64)
    { k_cast<float, double><<<grid, 256, 0, s>>>((const float*)src, lds, (double*)dst, ldd, rows, cols); ::sghsc::note_launch(); }
  else if (src_t == SG_F64 && dst_t == SG_F64)
    { k_cast<double, double><<<grid, 256, 0, s>>>((const double*)src, lds, (double*)dst, ldd, rows, cols); ::sghsc::note_launch(); }
  else
    { k_cast<float, float><<<grid, 256, 0, s>>>((const float*)src, lds, (float*)dst, ldd, rows, cols); ::sghsc::note_launch(); }
  SG_CHECK_LAUNCH();
  return SG_OK;
}

__device__ __forceinline__ void set_cond(const OuterArgs& a, bool v) {
  if (a.has_cond) cudaGraphSetConditional(a.cond, v ? 1u : 0u);
  if (a.flag) *a.flag = v;
}

// r = F - Y (Y may be null: r = F); F.F and r.r -> relative residual, it = 0
__global__ void __launch_bounds__(256) k_outer_init(long long N, const double* __restrict__ F,
                                                    const double* __restrict__ Y, double* __restrict__ r, OuterArgs a) {
  double s0 = 0.0, s1 = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double f = F[i];
    const double v = Y ? f - Y[i] : f;
    r[i] = v;
    s0 += f * f;
    s1 += v * v;
  }
  double ff, rr;
  if (outer_reduce_last(s0, s1, a, ff, rr) && threadIdx.x == 0) {
    a.sc[SC_FF] = ff;
    a.sc[SC_RR] = rr;
    const double rel = ff == 0.0 ? 0.0 : sqrt(rr / ff);   // non-finite values propagate
    a.sc[SC_REL] = rel;
    a.hist_res[0] = rel;
    a.ctl->it = 0;
    if (!(rel == rel)) atomicOr(a.status, ST_OUTER_BREAKDOWN);
    set_cond(a, rel > a.tol && a.maxit > 0);
  }
}

// z.r and z.q: beta (0 on the first iteration; flexible: z_{k+1}.(r_{k+1}-r_k)/(z_k.r_k)
// with r_{k+1} - r_k = -alpha_k q_k) and rho = z.r
template <typename TZ>
__device__ __forceinline__ void outer_dots(long long N, const TZ* __restrict__ z, const double* __restrict__ r,
                                           const double* __restrict__ q, const OuterArgs& a) {
  const int it = a.ctl->it;
  double s0 = 0.0, s1 = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double zv = widen<double>(z[i]);   // an FP32 z exactly, with integer operations
    s0 += zv * r[i];
    if (it > 0) s1 += zv * q[i];
  }
  double zr, zq;
  if (outer_reduce_last(s0, s1, a, zr, zq) && threadIdx.x == 0) {
    double beta = 0.0;
    if (it > 0) {
      beta = a.flexible ? (-a.sc[SC_ALPHA] * zq) / a.sc[SC_RHO] : zr / a.sc[SC_RHO];
      a.hist_beta[it - 1] = beta;
    }
    a.sc[SC_BETA] = beta;
    a.sc[SC_RHO] = zr;
    if (!(zr == zr) || !(beta == beta)) atomicOr(a.status, ST_OUTER_BREAKDOWN);
  }
}

__global__ void __launch_bounds__(256) k_outer_dots(long long N, const double* __restrict__ z,
                                                    const double* __restrict__ r, const double* __restrict__ q,
                                                    OuterArgs a) {
  outer_dots(N, z, r, q, a);
}
__global__ void __launch_bounds__(256) k_outer_dots32(long long N, const float* __restrict__ z,
                                                      const double* __restrict__ r, const double* __restrict__ q,
                                                      OuterArgs a) {
  outer_dots(N, z, r, q, a);
}

// x += alpha p_new; r -= alpha q; r.r -> relative residual, it += 1, loop condition
__global__ void __launch_bounds__(256) k_outer_update(long long N, const double* pA, const double* pB,
                                                      const double* __restrict__ q, double* __restrict__ x,
                                                      double* __restrict__ r, OuterArgs a) {
  const int it = a.ctl->it;
  const double* __restrict__ pnew = (it & 1) ? pA : pB;
  const double al = a.sc[SC_ALPHA];
  double s0 = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    x[i] += al * pnew[i];
    const double rv = r[i] - al * q[i];
    r[i] = rv;
    s0 += rv * rv;
  }
  double rr, unused;
  if (outer_reduce_last(s0, 0.0, a, rr, unused) && threadIdx.x == 0) {
    a.sc[SC_RR] = rr;
    const double rel = a.sc[SC_FF] == 0.0 ? 0.0 : sqrt(rr / a.sc[SC_FF]);
    a.sc[SC_REL] = rel;
    const int itn = it + 1;
    a.ctl->it = itn;
    a.hist_res[itn] = rel;
    const bool bad = !(rel == rel) || (*a.status & (ST_OUTER_BREAKDOWN | ST_INNER_NOT_SPD));
    if (!(rel == rel)) atomicOr(a.status, ST_OUTER_BREAKDOWN);
    set_cond(a, !bad && rel > a.tol && itn < a.maxit);
  }
}

// Schur-reduced iteration: p = z (first iteration) or z + beta p, in place
__global__ void __launch_bounds__(256) k_schur_p(long long N, const double* __restrict__ z, double* __restrict__ p,
                                                 OuterArgs a) {
  const bool first = a.ctl->it == 0;
  const double beta = first ? 0.0 : a.sc[SC_BETA];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    p[i] = first ? z[i] : z[i] + beta * p[i];
}

// Schur-reduced iteration: p . q and alpha = rho / (p . q) (as the fused
// product of the full system does in its epilogue)
__global__ void __launch_bounds__(256) k_schur_pq(long long N, const double* __restrict__ p,
                                                  const double* __restrict__ q, OuterArgs a) {
  double s0 = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    s0 += p[i] * q[i];
  double pq, unused;
  if (outer_reduce_last(s0, 0.0, a, pq, unused) && threadIdx.x == 0) {
    a.sc[SC_PQ] = pq;
    if (!(pq > 0.0)) {
      atomicOr(a.status, ST_OUTER_BREAKDOWN);
      a.sc[SC_ALPHA] = 0.0;
    } else {
      a.sc[SC_ALPHA] = a.sc[SC_RHO] / pq;
    }
    a.hist_alpha[a.ctl->it] = a.sc[SC_ALPHA];
  }
}

// true relative residual ||F - Y|| / ||F|| with Y = A x
__global__ void __launch_bounds__(256) k_outer_true(long long N, const double* __restrict__ F,
                                                    const double* __restrict__ Y, OuterArgs a) {
  double s0 = 0.0, s1 = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double f = F[i], v = f - Y[i];
    s0 += f * f;
    s1 += v * v;
  }
  double ff, rr;
  if (outer_reduce_last(s0, s1, a, ff, rr) && threadIdx.x == 0) a.sc[SC_TRUE] = ff == 0.0 ? 0.0 : sqrt(rr / ff);
}

int vec_grid(long long N) { return (int)std::max<long long>(1, std::min<long long>((N + 255) / 256, 152LL * 8)); }

}  // namespace sghsc
