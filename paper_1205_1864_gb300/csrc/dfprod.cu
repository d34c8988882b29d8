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

// Stage chunk cs..cs+nzc-1 (nzc <= DF_CH): values [k][e], inputs [j][e],
// slots e >= nzc zero. The input rows go column position by column position
// (no integer division), the loads of all slots of a position in flight
// before their stores.
template <typename TX>
__device__ __forceinline__ void df_stage(int cs, int nzc, int M1, const int* __restrict__ colidx,
                                         const df64* __restrict__ vals, const TX* __restrict__ X, int ldx, int wx,
                                         df64* Vt, float* Xt) {
  for (int k = threadIdx.x; k < M1; k += blockDim.x) {
#pragma unroll
    for (int e = 0; e < DF_CH; ++e) Vt[k * DF_CH + e] = e < nzc ? vals[(size_t)(cs + e) * M1 + k] : df64(0.f, 0.f);
  }
  int col[DF_CH];
#pragma unroll
  for (int e = 0; e < DF_CH; ++e) col[e] = e < nzc ? colidx[cs + e] : -1;
  for (int j = threadIdx.x; j < wx; j += blockDim.x) {
    float v[DF_CH];
#pragma unroll
    for (int e = 0; e < DF_CH; ++e) v[e] = col[e] >= 0 ? exact_float(X[(size_t)col[e] * ldx + j]) : 0.f;
#pragma unroll
    for (int e = 0; e < DF_CH; ++e) Xt[j * DF_CH + e] = v[e];
  }
}

// sum_e a[e] x[e] over the DF_CH slots (constant offsets)
__device__ __forceinline__ df64 df_dot9(const df64* __restrict__ a, const float* __restrict__ x) {
  df64 s = df_mul_f(a[0], x[0]);
#pragma unroll
  for (int e = 1; e < DF_CH; ++e) s += df_mul_f(a[e], x[e]);
  return s;
}

enum { DF_SUB = 0, DF_PLAIN = 1, DF_OUTER = 2 };

// MODE DF_SUB: a level product, Y = Yin - sum (Yin FP64, Y FP32), the
// difference in double-float, rounded once to FP32. DF_PLAIN: the full
// product, Y = sum (FP64, one add of the pair per output). DF_OUTER: the
// outer CG step (as k_outer_matvec): p_new = z + beta p_old, q = A z + beta
// q_old, p_new . q and alpha, with X = z (FP32, or FP64 storage of FP32
// values).
// Shared memory: pair sums Ss[npair], diagonal terms Ds[wy] (DIAG, by output
// column in natural order, so the lanes of a warp read consecutive inputs),
// the coefficient classes Ctab[ncls] (loaded once per block), then the
// staged chunk Vt, Xt. The packed couplings stay in global memory, read
// coalesced through L1 (in shared memory they held a block to one per SM at
// P = 1001).
template <int MAXO, bool DIAG, int MODE, typename TX, typename TY, int LB>
__global__ void __launch_bounds__(LB, LB <= 256 ? 4 : 2) k_df_pairs(
    int n, const int* __restrict__ rowptr, const int* __restrict__ colidx, const df64* __restrict__ vals, int M1,
    const TX* __restrict__ X, int ldx, int wx, int npair, const int* __restrict__ pk, const int* __restrict__ pj,
    const int* __restrict__ eptr, const int* __restrict__ eperm, const unsigned* __restrict__ ctr,
    const int* __restrict__ etb, const df64* __restrict__ ctab, int ncls, int wy, const double* __restrict__ Yin,
    int ldyin, TY* __restrict__ Y, int ldy, double* pA, double* pB, double* __restrict__ q, OuterArgs a) {
  constexpr bool OUTER = MODE == DF_OUTER;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  df64* Ss = reinterpret_cast<df64*>(smem_raw);
  df64* Ds = Ss + npair;
  df64* Ctab = Ds + (DIAG ? wy : 0);
  df64* Vt = Ctab + ncls;
  float* Xt = reinterpret_cast<float*>(Vt + (size_t)M1 * DF_CH);
  for (int t = threadIdx.x; t < ncls; t += blockDim.x) Ctab[t] = ctab[t];
  // this thread's pairs (consecutive threads: consecutive pairs) and outputs
  unsigned qkj[DF_MAXQ];   // k << 16 | j
#pragma unroll
  for (int i = 0; i < DF_MAXQ; ++i) {
    const int qi = threadIdx.x + i * blockDim.x;
    qkj[i] = qi < npair ? ((unsigned)pk[qi] << 16) | (unsigned)pj[qi] : 0u;
  }
  // the couplings of this thread's outputs: slot-transposed in global memory
  // (the table is the same for every block and row, so it stays in L1)
  int lcol[MAXO], t0[MAXO], nc[MAXO];
#pragma unroll
  for (int i = 0; i < MAXO; ++i) {
    const int slot = threadIdx.x + i * blockDim.x;
    lcol[i] = slot < wy ? eperm[slot] : -1;
    t0[i] = lcol[i] >= 0 ? etb[slot] : 0;
    nc[i] = lcol[i] >= 0 ? eptr[lcol[i] + 1] - eptr[lcol[i]] : 0;
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
#pragma unroll
        for (int i = 0; i < MAXO; ++i) {
          const int l = threadIdx.x + i * blockDim.x;
          if (l < wy) {
            const df64 d = df_dot9(Vt, Xt + l * DF_CH);
            if (first) Ds[l] = d; else Ds[l] += d;
          }
        }
      }
#pragma unroll
      for (int i = 0; i < DF_MAXQ; ++i) {
        const int qi = threadIdx.x + i * blockDim.x;
        if (qi < npair) {
          const df64 s = df_dot9(Vt + (qkj[i] >> 16) * DF_CH, Xt + (qkj[i] & 0xffffu) * DF_CH);
          if (first) Ss[qi] = s; else Ss[qi] += s;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < MAXO; ++i) {
      const int l = lcol[i];
      if (l < 0) continue;
      df64 acc = (DIAG && re > rb) ? Ds[l] : df64(0.f, 0.f);
      if (re > rb) {
        const unsigned* cw = ctr + t0[i];
#pragma unroll 4
        for (int c = 0; c < nc[i]; ++c) {
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

static size_t df_smem(const EdgeList& E, int M1, int wx, bool diag) {
  return ((size_t)E.npair + (diag ? E.nout : 0) + E.ncls + (size_t)M1 * DF_CH) * sizeof(df64) +
         (size_t)wx * DF_CH * sizeof(float);
}

// Block size: 256 threads when the pairs and two outputs per thread fit, else
// 512 (more, smaller blocks hide the row barriers better; more outputs per
// thread would spill).
static int df_threads(const EdgeList& E) { return E.npair <= DF_MAXQ * 256 && E.nout <= 512 ? 256 : 512; }

// Usable when every thread's pairs fit its registers, the couplings have a
// compact table and the staging fits a block's shared memory.
bool df_pairs_usable(const sg_problem* h, const EdgeList& E, int wx) {
  return h->staged_pairs && E.npair <= DF_MAXQ * 512 && E.ncls > 0 && h->nterm < 65536 && wx < 65536 &&
         df_smem(E, h->nterm, wx, true) <= (size_t)std::max(h->smem_optin, 48 * 1024);
}

template <bool DIAG, int MODE, typename TX, typename TY>
static int launch_df(sg_problem* h, const EdgeList& E, const TX* X, int ldx, int wx, const double* Yin, int ldyin,
                     TY* Y, int ldy, const OuterArgs* oa, cudaStream_t s) {
  const int wy = E.nout;
  if (wy == 0) return SG_OK;
  const int threads = df_threads(E);
  const int maxo = (wy + threads - 1) / threads;
  const size_t smem = df_smem(E, h->nterm, wx, DIAG);
  OuterArgs a = oa ? *oa : OuterArgs{};
  auto go = [&](auto kern) -> int {
    SG_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    int grid = std::min(h->n, h->num_sms * std::max(per_sm, 1));
    if (MODE == DF_OUTER) grid = std::min(grid, h->opart_blocks);
    { kern<<<grid, threads, smem, s>>>(h->n, h->rowptr, h->colidx, (const df64*)h->vals_df, h->nterm, X, ldx, wx,
                                       E.npair, E.pk, E.pj, E.ptr, E.perm, E.ctr, E.tb, (const df64*)E.ctab, E.ncls,
                                       wy, Yin, ldyin, Y, ldy, h->fpA, h->fpB, h->fq, a); ::sghsc::note_launch(); }
    SG_CHECK_LAUNCH();
    return SG_OK;
  };
  if (threads == 256) {
    if (maxo <= 1) return go(k_df_pairs<1, DIAG, MODE, TX, TY, 256>);
    if (maxo <= 2) return go(k_df_pairs<2, DIAG, MODE, TX, TY, 256>);
  } else {
    if (maxo <= 1) return go(k_df_pairs<1, DIAG, MODE, TX, TY, 512>);
    if (maxo <= 2) return go(k_df_pairs<2, DIAG, MODE, TX, TY, 512>);
    if (maxo <= 4) return go(k_df_pairs<4, DIAG, MODE, TX, TY, 512>);
  }
  set_error("double-float product: %d outputs exceed the supported 2048", wy);
  return SG_ERR_UNSUPPORTED;
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
