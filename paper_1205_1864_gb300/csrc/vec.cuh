// Outer-solver kernels shared by the FCG driver (vec.cu, matvec.cu, fcg.cu).
#pragma once

#include "sghsc_internal.cuh"

namespace sghsc {

// Slots of the device scalar array of the outer solver.
enum { SC_RHO = 0, SC_PQ, SC_ALPHA, SC_BETA, SC_RR, SC_FF, SC_REL, SC_TRUE, SC_COUNT };

// Arguments of the outer kernels that finish with a last-block update of the
// CG scalars (passed by value).
struct OuterArgs {
  double* part;             // [nblk][2] block partials
  OuterCtl* ctl;
  double* sc;               // SC_* scalars
  double *hist_alpha, *hist_beta, *hist_res;
  int* status;
  int flexible;
  int maxit;
  double tol;
  cudaGraphConditionalHandle cond;
  int has_cond;
  int* flag;
};

__global__ void k_outer_init(long long N, const double* F, const double* Y, double* r, OuterArgs a);
__global__ void k_outer_dots(long long N, const double* z, const double* r, const double* q, OuterArgs a);
// the same with the FP32 z of the mixed preconditioners
__global__ void k_outer_dots32(long long N, const float* z, const double* r, const double* q, OuterArgs a);
__global__ void k_outer_update(long long N, const double* pA, const double* pB, const double* q, double* x,
                               double* r, OuterArgs a);
__global__ void k_outer_true(long long N, const double* F, const double* Y, OuterArgs a);
__global__ void k_schur_p(long long N, const double* z, double* p, OuterArgs a);
__global__ void k_schur_pq(long long N, const double* p, const double* q, OuterArgs a);

// Fixed-order tree sum of r0[0 .. blockDim), r1[...] into r0[0], r1[0]:
// the entries above the largest power of two p2 <= blockDim are first added
// to entries 0 .. blockDim - p2 (nothing for a power-of-two block), then the
// halving tree over p2 entries.
__device__ __forceinline__ void tree_sum2(double* r0, double* r1) {
  int p2 = 1;
  while (2 * p2 <= (int)blockDim.x) p2 *= 2;
  if (p2 < (int)blockDim.x) {
    if ((int)threadIdx.x < (int)blockDim.x - p2) {
      r0[threadIdx.x] += r0[threadIdx.x + p2];
      r1[threadIdx.x] += r1[threadIdx.x + p2];
    }
    __syncthreads();
  }
  for (int s = p2 / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      r0[threadIdx.x] += r0[threadIdx.x + s];
      r1[threadIdx.x] += r1[threadIdx.x + s];
    }
    __syncthreads();
  }
}

// Fixed-order block sum of (v0, v1) to part[blockIdx]; returns true in the last
// block, whose threads then hold the totals (t0, t1) over all blocks (summed in
// block order). blockDim <= 1024.
__device__ __forceinline__ bool outer_reduce_last(double v0, double v1, const OuterArgs& a, double& t0, double& t1) {
  __shared__ double r0[1024], r1[1024];
  __shared__ bool last;
  r0[threadIdx.x] = v0;
  r1[threadIdx.x] = v1;
  __syncthreads();
  tree_sum2(r0, r1);
  if (threadIdx.x == 0) {
    a.part[(size_t)blockIdx.x * 2 + 0] = r0[0];
    a.part[(size_t)blockIdx.x * 2 + 1] = r1[0];
    __threadfence();
    last = atomicAdd(&a.ctl->ticket, 1u) == gridDim.x - 1;
    if (last) __threadfence();
  }
  __syncthreads();
  if (!last) return false;
  double s0 = 0.0, s1 = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    s0 += __ldcg(&a.part[(size_t)b * 2 + 0]);
    s1 += __ldcg(&a.part[(size_t)b * 2 + 1]);
  }
  r0[threadIdx.x] = s0;
  r1[threadIdx.x] = s1;
  __syncthreads();
  tree_sum2(r0, r1);
  t0 = r0[0];
  t1 = r1[0];
  if (threadIdx.x == 0) a.ctl->ticket = 0;
  return true;
}


// Exact FP32 -> FP64 conversion from the IEEE-754 layouts, integer operations
// only (the FP64 pipe of this GPU is narrow, and a hardware conversion issues
// there): sign kept; a normal number's exponent rebiased by 1023 - 127 and its
// 23-bit fraction shifted into the top of the 52-bit one; a subnormal m 2^-149
// (m < 2^23) renormalised from its leading one at bit q: exponent q - 149 +
// 1023, fraction m shifted so that bit q lands just above bit 51 (dropped);
// zeros, infinities and NaNs keep their classes.
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  unsigned long long bits;
  if (e == 0u && m != 0u) {
    const unsigned q = 31u - (unsigned)__clz(m);
    bits = sign | ((unsigned long long)(q + 874u) << 52) | (((unsigned long long)m << (52u - q)) & 0xfffffffffffffull);
  } else {
    const unsigned ed = e == 0u ? 0u : (e == 0xffu ? 0x7ffu : e + 896u);
    bits = sign | ((unsigned long long)ed << 52) | ((unsigned long long)m << 29);
  }
  return __longlong_as_double((long long)bits);
}

// v converted to TD; float -> double through f2d_bits.
template <typename TD, typename TS>
__device__ __forceinline__ TD widen(TS v) {
  if constexpr (sizeof(TD) == 8 && sizeof(TS) == 4) return f2d_bits(v);
  else return (TD)v;
}

// Asynchronous global -> shared copy of one 4- or 8-byte element (cp.async,
// completed by cp_async_wait_all); all of a block's copies are in flight
// together instead of one load latency per element.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

int vec_grid(long long N);

// The outer CG step q = A p_new with p_new = z + beta p_old staged on the fly
// (ping-pong p buffers chosen by the device iteration counter), the fused
// p_new . q reduction and the alpha update by the last block (matvec.cu).
// df: the product in double-float arithmetic on the FP32 units (z32: the
// preconditioned residual in FP32 when the preconditioner leaves it there).
int launch_outer_matvec(sg_problem* h, const OuterArgs& a, cudaStream_t s, bool df = false,
                        const float* z32 = nullptr);
// The same in the double-float pair form (dfprod.cu); z must hold FP32 values,
// which z32 (n x P FP32, or null: read z) holds as well.
int launch_df_outer(sg_problem* h, const OuterArgs& a, cudaStream_t s, const float* z32);
// Arguments of the outer-iteration kernels for this handle and options (fcg.cu).
OuterArgs outer_args(sg_problem* h, const sg_solve_opts& o);

}  // namespace sghsc
