// Double-float SG products whose input block holds FP32 values (the output
// of the mixed-precision preconditioner): the outer solver's fused product
// q = A p (eq. (global-system) in MAT-VEC form, with the CG update) and the
// level-p products B_p, C_p of Algorithm 1. The arithmetic is double-float
// (df64.cuh) on the FP32 units; this file lays the work out for those units.
//
// Pair form, one spatial row at a time per block (grid-stride over rows):
//   stage   the row's values a_k(r, c) as [k][e] and the input rows X(c, :)
//           as [j][e] (e the nonzero, CH = 9 slots, zero-filled), so the
//           inner loop over the 9 nonzeros uses constant offsets only and the
//           lanes of a warp (consecutive pairs: the same k, consecutive j)
//           read one broadcast value and 32 distinct banks (stride 9 words);
//   pairs   every distinct (k, j) of the couplings: S_q = sum_e a_k(e) X(e, j)
//           into shared memory, each thread keeping its pairs in registers;
//           with DIAG also the k = 0 term of its own outputs;
//   couple  Y(r, l) = diag + sum_t c_t S_pair(t) over the couplings of l.
// Rows longer than CH are done in chunks of CH (the first chunk stores, later
// ones add).
#include <algorithm>
#include <type_traits>

#include "df64.cuh"
#include "sghsc_internal.cuh"
#include "vec.cuh"

namespace sghsc {

constexpr int DF_CH = 9;       // nonzeros per staged chunk (the Q1 stencil row)
constexpr int DF_MAXQ = 12;    // pairs per thread kept in registers

// FP32 value of an input element that is FP32-exact: a float as it is, a
// double (the FP64 widening of an FP32 number) re-packed with integer
// operations (truncating the fraction, which is exact for such values).
__device__ __forceinline__ float exact_float(float v) { return v; }
__device__ __forceinline__ float exact_float(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int E = (int)((b >> 52) & 0x7ff);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  if (E == 0) return __uint_as_float(sign);
  const int ef = E - 1023 + 127;
  if (ef < 1 || ef > 254) return __double2float_rn(v);   // outside the normal FP32 range (not expected)
  return __uint_as_float(sign | ((unsigned)ef << 23) | (unsigned)((b >> 29) & 0x7fffffu));
}

// an input element as FP64: a float widened with integer operations, a double as it is
__device__ __forceinline__ double widen_exact(float v) { return f2d_bits(v); }
__device__ __forceinline__ double widen_exact(double v) { return v; }

// a (double-float) times x (FP32): exact product of a.hi and x plus a.lo x
__device__ __forceinline__ df64 df_mul_f(const df64& a, float x) {
  const float p = a.hi * x;
  float e = fmaf(a.hi, x, -p);
  e = fmaf(a.lo, x, e);
  return df64(p, e);
}

// Row strides of the staged chunk: a term's nine values padded to ten
// double-float slots (80 bytes: five 16-byte loads), an input column's nine
// values padded to twelve floats (48 bytes: three 16-byte loads; a warp's
// eight-lane phases of consecutive columns then hit distinct bank groups).
constexpr int DF_VS = 10;
constexpr int DF_XS = 12;

// Stage chunk cs..cs+nzc-1 (nzc <= DF_CH): values [k][e], inputs [j][e],
// slots e >= nzc zero. The input rows go column position by column position
// (no integer division), the loads of all slots of a position in flight
// before their 16-byte stores.
template <typename TX>
__device__ __forceinline__ void df_stage(int cs, int nzc, int M1, const int* __restrict__ colidx,
                                         const df64* __restrict__ vals, const TX* __restrict__ X, int ldx, int wx,
                                         df64* Vt, float* Xt) {
  for (int k = threadIdx.x; k < M1; k += blockDim.x) {
#pragma unroll
    for (int e = 0; e < DF_VS; ++e) Vt[k * DF_VS + e] = e < nzc ? vals[(size_t)(cs + e) * M1 + k] : df64(0.f, 0.f);
  }
  int col[DF_CH];
#pragma unroll
  for (int e = 0; e < DF_CH; ++e) col[e] = e < nzc ? colidx[cs + e] : -1;
  for (int j = threadIdx.x; j < wx; j += blockDim.x) {
    float v[DF_CH];
#pragma unroll
    for (int e = 0; e < DF_CH; ++e) v[e] = col[e] >= 0 ? exact_float(X[(size_t)col[e] * ldx + j]) : 0.f;
    float4* xr = reinterpret_cast<float4*>(Xt + j * DF_XS);
    xr[0] = make_float4(v[0], v[1], v[2], v[3]);
    xr[1] = make_float4(v[4], v[5], v[6], v[7]);
    xr[2] = make_float4(v[8], 0.f, 0.f, 0.f);
  }
}

// sum_e a[e] x[e] over the DF_CH slots of one staged term row and one staged
// input column, both read as 16-byte vectors
__device__ __forceinline__ df64 df_dot9(const df64* __restrict__ a, const float* __restrict__ x) {
  const float4* av = reinterpret_cast<const float4*>(a);   // two double-float values each
  const float4* xv = reinterpret_cast<const float4*>(x);
  const float4 x0 = xv[0], x1 = xv[1], x2 = xv[2];
  float4 v = av[0];
  df64 s = df_mul_f(df64(v.x, v.y), x0.x);
  s += df_mul_f(df64(v.z, v.w), x0.y);
  v = av[1];
  s += df_mul_f(df64(v.x, v.y), x0.z);
  s += df_mul_f(df64(v.z, v.w), x0.w);
  v = av[2];
  s += df_mul_f(df64(v.x, v.y), x1.x);
  s += df_mul_f(df64(v.z, v.w), x1.y);
  v = av[3];
  s += df_mul_f(df64(v.x, v.y), x1.z);
  s += df_mul_f(df64(v.z, v.w), x1.w);
  v = av[4];
  s += df_mul_f(df64(v.x, v.y), x2.x);
  return s;
}

enum { DF_SUB = 0, DF_PLAIN = 1, DF_OUTER = 2 };

// MODE DF_SUB: a level product, Y = Yin - sum (Yin FP64, Y FP32), the
// difference in double-float, rounded once to FP32. DF_PLAIN: the full
// product, Y = sum (FP64, one add of the pair per output). DF_OUTER: the
// outer CG step (as k_outer_matvec): p_new = z + beta p_old, q = A z + beta
// q_old, p_new . q and alpha, with X = z (FP32, or FP64 storage of FP32
// values).
// Shared memory (16-byte aligned parts): pair sums Ss[npair], diagonal terms
// Ds[wy] (DIAG, by output column in natural order, so the lanes of a warp
// read consecutive inputs), the coefficient classes Ctab[ncls] (loaded once
// per block), then the staged chunk Vt, Xt. The packed couplings stay in
// global memory, read coalesced through L1 (in shared memory they held a
// block to one per SM at P = 1001); each output slot's first word and count
// come from a descriptor, so a thread takes any number of outputs.
template <bool DIAG, int MODE, typename TX, typename TY, int LB>
__global__ void __launch_bounds__(LB, LB <= 256 ? 4 : 2) k_df_pairs(
    int n, const int* __restrict__ rowptr, const int* __restrict__ colidx, const df64* __restrict__ vals, int M1,
    const TX* __restrict__ X, int ldx, int wx, int npair, const int* __restrict__ pk, const int* __restrict__ pj,
    const unsigned* __restrict__ ctr, const int2* __restrict__ sdesc, const df64* __restrict__ ctab, int ncls, int wy,
    const double* __restrict__ Yin, int ldyin, TY* __restrict__ Y, int ldy, double* pA, double* pB,
    double* __restrict__ q, OuterArgs a) {
  constexpr bool OUTER = MODE == DF_OUTER;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // pairs and diagonal outputs padded to whole passes of the block, so every
  // warp runs the same loops (the padding pairs read staged slot 0 and write
  // sums nothing reads)
  const int nq = (npair + LB - 1) / LB, nd = DIAG ? (wy + LB - 1) / LB : 0;
  df64* Ss = reinterpret_cast<df64*>(smem_raw);
  df64* Ds = Ss + (size_t)nq * LB;
  df64* Ctab = Ds + (size_t)nd * LB;
  df64* Vt = Ctab + ((ncls + 1) & ~1);
  float* Xt = reinterpret_cast<float*>(Vt + (size_t)M1 * DF_VS);
  for (int t = threadIdx.x; t < ncls; t += blockDim.x) Ctab[t] = ctab[t];
  // this thread's pairs (consecutive threads: consecutive pairs), as the
  // staged offsets of their term row and input column
  unsigned qkj[DF_MAXQ];   // k DF_VS << 16 | j DF_XS
#pragma unroll
  for (int i = 0; i < DF_MAXQ; ++i) {
    const int qi = threadIdx.x + i * blockDim.x;
    qkj[i] = qi < npair ? ((unsigned)(pk[qi] * DF_VS) << 16) | (unsigned)(pj[qi] * DF_XS) : 0u;
  }
  int it = 0;
  double beta = 0.0, dot = 0.0;
  const double* pold = nullptr;
  double* pnew = nullptr;
  if constexpr (OUTER) {
    it = a.ctl->it;
    beta = it == 0 ? 0.0 : a.sc[SC_BETA];
    pold = (it & 1) ? pB : pA;
    pnew = (it & 1) ? pA : pB;
  }
  for (int r = blockIdx.x; r < n; r += gridDim.x) {
    const int rb = rowptr[r], re = rowptr[r + 1];
    for (int cs = rb; cs < re; cs += DF_CH) {
      const int nzc = min(DF_CH, re - cs);
      __syncthreads();
      df_stage<TX>(cs, nzc, M1, colidx, vals, X, ldx, wx, Vt, Xt);
      __syncthreads();
      const bool first = cs == rb;
      if (DIAG) {
        for (int i = 0; i < nd; ++i) {
          const int l = threadIdx.x + i * LB;
          const df64 d = df_dot9(Vt, Xt + min(l, wx - 1) * DF_XS);
          if (first) Ds[l] = d; else Ds[l] += d;
        }
      }
#pragma unroll
      for (int i = 0; i < DF_MAXQ; ++i) {
        if (i < nq) {   // the same for the whole block
          const int qi = threadIdx.x + i * LB;
          const df64 s = df_dot9(Vt + (qkj[i] >> 16), Xt + (qkj[i] & 0xffffu));
          if (first) Ss[qi] = s; else Ss[qi] += s;
        }
      }
    }
    __syncthreads();
    for (int slot = threadIdx.x; slot < wy; slot += LB) {
      const int2 d = __ldg(sdesc + slot);
      const int l = (int)((unsigned)d.y >> 16), ncl = d.y & 0xffff;   // ncl: the warp's count
      df64 acc = (DIAG && re > rb) ? Ds[l] : df64(0.f, 0.f);
      if (re > rb) {
        const unsigned* cw = ctr + d.x;
#pragma unroll 4
        for (int c = 0; c < ncl; ++c) {
          const unsigned w = __ldg(cw + 32 * c);
          acc += Ctab[w & 0xffu] * Ss[w >> 8];
        }
      }
      acc = df_norm(acc);
      if constexpr (OUTER) {
        const size_t g = (size_t)r * wx + l;
        const double av = f2d_bits(acc.hi) + f2d_bits(acc.lo);
        const double zv = widen_exact(X[g]);
        const double pv = it == 0 ? zv : zv + beta * pold[g];
        const double qv = it == 0 ? av : av + beta * q[g];
        pnew[g] = pv;
        q[g] = qv;
        dot += pv * qv;
      } else if constexpr (MODE == DF_PLAIN) {
        Y[(size_t)r * ldy + l] = f2d_bits(acc.hi) + f2d_bits(acc.lo);
      } else {
        // Yin - sum in double-float, rounded once to FP32
        df64 v = df_from_double(Yin[(size_t)r * ldyin + l]);
        v += df64(-acc.hi, -acc.lo);
        Y[(size_t)r * ldy + l] = v.hi + v.lo;
      }
    }
  }
  if constexpr (OUTER) {
    double pq, unused;
    if (outer_reduce_last(dot, 0.0, a, pq, unused) && threadIdx.x == 0) {
      a.sc[SC_PQ] = pq;
      if (!(pq > 0.0)) {
        atomicOr(a.status, ST_OUTER_BREAKDOWN);
        a.sc[SC_ALPHA] = 0.0;
      } else {
        a.sc[SC_ALPHA] = a.sc[SC_RHO] / pq;
      }
      a.hist_alpha[it] = a.sc[SC_ALPHA];
    }
  }
}

// Block size: 256 threads when every thread's pairs fit its registers, else
// 512 (more, smaller blocks hide the row barriers better).
static int df_threads(const EdgeList& E) { return E.npair <= DF_MAXQ * 256 ? 256 : 512; }

static size_t df_smem(const EdgeList& E, int M1, int wx, bool diag) {
  const size_t t = (size_t)df_threads(E);
  auto pad = [t](size_t v) { return (v + t - 1) / t * t; };
  return (pad(E.npair) + (diag ? pad(E.nout) : 0) + ((E.ncls + 1) & ~1) + (size_t)M1 * DF_VS) * sizeof(df64) +
         (size_t)wx * DF_XS * sizeof(float);
}

// Usable when every thread's pairs fit its registers, the couplings have a
// compact table with slot descriptors and the staging fits a block's shared
// memory.
bool df_pairs_usable(const sg_problem* h, const EdgeList& E, int wx) {
  return h->staged_pairs && E.npair <= DF_MAXQ * 512 && E.ncls > 0 && E.sdesc && h->nterm * DF_VS < 65536 &&
         wx * DF_XS < 65536 && df_smem(E, h->nterm, wx, true) <= (size_t)std::max(h->smem_optin, 48 * 1024);
}

template <bool DIAG, int MODE, typename TX, typename TY>
static int launch_df(sg_problem* h, const EdgeList& E, const TX* X, int ldx, int wx, const double* Yin, int ldyin,
                     TY* Y, int ldy, const OuterArgs* oa, cudaStream_t s) {
  const int wy = E.nout;
  if (wy == 0) return SG_OK;
  const int threads = df_threads(E);
  const size_t smem = df_smem(E, h->nterm, wx, DIAG);
  OuterArgs a = oa ? *oa : OuterArgs{};
  auto go = [&](auto kern) -> int {
    SG_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    int grid = std::min(h->n, h->num_sms * std::max(per_sm, 1));
    if (MODE == DF_OUTER) grid = std::min(grid, h->opart_blocks);
    { kern<<<grid, threads, smem, s>>>(h->n, h->rowptr, h->colidx, (const df64*)h->vals_df, h->nterm, X, ldx, wx,
                                       E.npair, E.pk, E.pj, E.ctr, E.sdesc, (const df64*)E.ctab, E.ncls, wy, Yin,
                                       ldyin, Y, ldy, h->fpA, h->fpB, h->fq, a); ::sghsc::note_launch(); }
    SG_CHECK_LAUNCH();
    return SG_OK;
  };
  if (threads == 256) return go(k_df_pairs<DIAG, MODE, TX, TY, 256>);
  return go(k_df_pairs<DIAG, MODE, TX, TY, 512>);
}

int launch_df_level(sg_problem* h, const EdgeList& E, const float* X, int ldx, int wx, const double* Yin, int ldyin,
                    float* Y, int ldy, cudaStream_t s) {
  return launch_df<false, DF_SUB, float, float>(h, E, X, ldx, wx, Yin, ldyin, Y, ldy, nullptr, s);
}

int launch_df_outer(sg_problem* h, const OuterArgs& a, cudaStream_t s, const float* z32) {
  // z itself in FP32 when the preconditioner leaves it there (half the staging reads, no conversion)
  float* none = nullptr;
  if (z32) return launch_df<true, DF_OUTER, float, float>(h, h->all, z32, h->P, h->P, nullptr, 0, none, 0, &a, s);
  return launch_df<true, DF_OUTER, double, float>(h, h->all, h->fz, h->P, h->P, nullptr, 0, none, 0, &a, s);
}

int launch_df_apply(sg_problem* h, const float* U, double* Y, cudaStream_t s) {
  return launch_df<true, DF_PLAIN, float, double>(h, h->all, U, h->P, h->P, nullptr, 0, Y, h->P, nullptr, s);
}

}  // namespace sghsc
