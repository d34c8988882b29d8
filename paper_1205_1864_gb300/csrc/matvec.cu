// K1 (fused SG matrix-vector product, eq. (global-system) in MAT-VEC form)
// and K2 (off-diagonal level products B_l, C_l of Algorithm 1).
//
// One thread block owns one spatial row r at a time (grid-stride over rows,
// consecutive blocks on consecutive rows so the 9 neighbour rows of U are
// shared through L2). For each chunk of the row's nonzeros it stages the
// neighbour rows U(c, :) and the M+1 values a_k(r, c) of every nonzero in
// shared memory -- the shared CSR pattern is read once and all KL matrices
// ride along -- and each thread then forms its output columns l by the
// gather form of the sparse G couplings:
//   Y(r,l) = sum_c a_0(r,c) U(c,l) + sum_{(k,j): alpha_j = alpha_l +- e_k}
//            (G_k)_{lj} sum_c a_k(r,c) U(c,j).
// Per nonzero that is P + n_m multiply-adds (n_m the off-diagonal G entries),
// the smallest count of the contraction orders; the full product sums each
// distinct (k, j) once (pair form below), P + npair per nonzero plus n_m per
// row.
#include <algorithm>
#include <type_traits>

#include "df64.cuh"
#include "sghsc_internal.cuh"
#include "vec.cuh"

namespace sghsc {

// An input element in the accumulation type: FP32 -> FP64 by integer
// widening, FP32/FP64 -> double-float by exact splitting (no FP64 operation).
template <typename TAcc, typename TIn>
__device__ __forceinline__ TAcc to_acc(TIn v) {
  if constexpr (std::is_same_v<TAcc, df64>) {
    if constexpr (sizeof(TIn) == 4) return df_from_float(v);
    else return df_from_double(v);
  } else {
    return widen<TAcc>(v);
  }
}

// An accumulated value as FP64 (double-float: two integer widenings, one add).
template <typename TAcc>
__device__ __forceinline__ double acc_to_double(const TAcc& v) {
  if constexpr (std::is_same_v<TAcc, df64>) {
    const df64 x = df_norm(v);
    return f2d_bits(x.hi) + f2d_bits(x.lo);
  } else {
    return (double)v;
  }
}

// This thread's output columns: slot threadIdx + i * blockDim takes column
// eperm[slot] (outputs ordered by coupling count, so the lanes of a warp run
// coupling loops of equal length); -1 past the last output.
template <int MAXO>
__device__ __forceinline__ void output_columns(const int* __restrict__ eperm, int wy, int (&lcol)[MAXO]) {
#pragma unroll
  for (int i = 0; i < MAXO; ++i) {
    const int slot = threadIdx.x + i * blockDim.x;
    lcol[i] = slot < wy ? eperm[slot] : -1;
  }
}

// Stage the chunk of nzc nonzeros starting at cs: the neighbour rows X(c, :)
// (widened to TAcc) and the M+1 values of each nonzero. Same-type rows and
// the values go by asynchronous copies (all in flight at once); a widened row
// by batches of 4 loads in flight before the conversions. The caller waits
// (cp_async_wait_all) and synchronises.
template <typename TIn, typename TAcc>
__device__ __forceinline__ void stage_chunk(int cs, int nzc, int M1, const int* __restrict__ colidx,
                                            const TAcc* __restrict__ vals, const TIn* __restrict__ X, int ldx,
                                            int wx, TAcc* Xs, TAcc* Vs) {
  const int cnt = nzc * wx;
  if constexpr (std::is_same_v<TIn, TAcc>) {
    for (int idx = threadIdx.x; idx < cnt; idx += blockDim.x) {
      const int e = idx / wx, j = idx - e * wx;
      cp_async_elem(Xs + idx, X + (size_t)colidx[cs + e] * ldx + j);
    }
  } else {
    for (int base = threadIdx.x; base < cnt; base += 4 * blockDim.x) {
      TIn v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int idx = base + u * blockDim.x;
        if (idx < cnt) {
          const int e = idx / wx, j = idx - e * wx;
          v[u] = X[(size_t)colidx[cs + e] * ldx + j];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int idx = base + u * blockDim.x;
        if (idx < cnt) Xs[idx] = to_acc<TAcc>(v[u]);
      }
    }
  }
  for (int idx = threadIdx.x; idx < nzc * M1; idx += blockDim.x) cp_async_elem(Vs + idx, vals + (size_t)cs * M1 + idx);
}

// Accumulate the gather form for this thread's outputs over one staged chunk
// (a level product names every pair (k, j) once: this is its form). FIRST:
// the row's first chunk stores its sums (no FP64 add of a zero).
template <typename TAcc, int MAXO, bool DIAG, bool FIRST>
__device__ __forceinline__ void gather_chunk(int nzc, int M1, const TAcc* __restrict__ Vs,
                                             const TAcc* __restrict__ Xs, int wx, const int* __restrict__ eptr,
                                             const int* __restrict__ ek, const int* __restrict__ ej,
                                             const TAcc* __restrict__ ec, const int (&lcol)[MAXO],
                                             TAcc (&acc)[MAXO]) {
#pragma unroll
  for (int i = 0; i < MAXO; ++i) {
    const int l = lcol[i];
    if (l >= 0) {
      TAcc a = TAcc(0);
      if (DIAG) {
        for (int e = 0; e < nzc; ++e) a += Vs[e * M1] * Xs[e * wx + l];
      }
      const int t1 = eptr[l + 1];
      for (int t = eptr[l]; t < t1; ++t) {
        const int k = ek[t], j = ej[t];
        TAcc s = TAcc(0);
        for (int e = 0; e < nzc; ++e) s += Vs[e * M1 + k] * Xs[e * wx + j];
        a += ec[t] * s;
      }
      if (FIRST)
        acc[i] = a;
      else
        acc[i] += a;
    }
  }
}

// The full SG product in pair form (DIAG): per staged chunk, the diagonal
// term of this thread's outputs into acc, and for every distinct pair
// q = (k, j) of the couplings s_q = sum_c a_k(r,c) U(c,j) into Ss (FIRST: the
// row's first chunk stores, later ones add). A pair serves every coupling that
// names it (an input column j coupled to two outputs in direction k is summed
// once), so this does 9 (P + npair) multiply-adds per 9-point row instead of
// 9 (P + n_m); consecutive pairs share k and take consecutive j. It needs
// npair more values of shared memory, which can cost resident blocks: the
// autotuner times both forms.
template <typename TAcc, int MAXO, bool FIRST>
__device__ __forceinline__ void pair_chunk(int nzc, int M1, const TAcc* __restrict__ Vs, const TAcc* __restrict__ Xs,
                                           int wx, int npair, const int* __restrict__ pk,
                                           const int* __restrict__ pj, TAcc* Ss, const int (&lcol)[MAXO],
                                           TAcc (&acc)[MAXO]) {
#pragma unroll
  for (int i = 0; i < MAXO; ++i) {
    const int l = lcol[i];
    if (l >= 0) {
      TAcc a = TAcc(0);
      for (int e = 0; e < nzc; ++e) a += Vs[e * M1] * Xs[e * wx + l];
      if (FIRST)
        acc[i] = a;
      else
        acc[i] += a;
    }
  }
  for (int q = threadIdx.x; q < npair; q += blockDim.x) {
    const int k = pk[q], j = pj[q];
    TAcc s = TAcc(0);
    for (int e = 0; e < nzc; ++e) s += Vs[e * M1 + k] * Xs[e * wx + j];
    if (FIRST)
      Ss[q] = s;
    else
      Ss[q] += s;
  }
}

// After the row's last chunk and a block barrier: the couplings of this
// thread's outputs from the pair sums, in coupling order.
template <typename TAcc, int MAXO>
__device__ __forceinline__ void pair_couple(const int* __restrict__ eptr, const int* __restrict__ pair,
                                            const TAcc* __restrict__ ec, const TAcc* Ss, const int (&lcol)[MAXO],
                                            TAcc (&acc)[MAXO]) {
#pragma unroll
  for (int i = 0; i < MAXO; ++i) {
    const int l = lcol[i];
    if (l >= 0) {
      TAcc a = acc[i];
      const int t1 = eptr[l + 1];
      for (int t = eptr[l]; t < t1; ++t) a += ec[t] * Ss[pair[t]];
      acc[i] = a;
    }
  }
}

// alpha, beta of the product's epilogue: a test against a small integer and the
// value in FP64 (double-float scalars carry their value in hi).
template <typename T>
__device__ __forceinline__ bool is_value(const T& x, float v) {
  if constexpr (std::is_same_v<T, df64>) return x.hi == v && x.lo == 0.f;
  else return x == (T)v;
}
__device__ __forceinline__ double df_to_scale(const df64& x) { return f2d_bits(x.hi) + f2d_bits(x.lo); }

// LB: the largest block the instantiation is launched with. Blocks of up to
// 256 threads with fewer than 4 outputs per thread keep the compiler's
// register choice; with 4 or more (large P) they may use up to 64 registers
// (4 blocks per SM) instead of spilling; blocks of up to 1024 threads may use
// 64 (one block per SM).
#define SG_MATVEC_BOUNDS(LB, MAXO) __launch_bounds__(LB, (LB) > 256 ? 1 : ((MAXO) >= 4 ? 4 : 0))

template <typename TIn, typename TAcc, typename TB, typename TO, bool DIAG, int MAXO, int LB>
__global__ void SG_MATVEC_BOUNDS(LB, MAXO) k_block_matvec(
    int n, const int* __restrict__ rowptr, const int* __restrict__ colidx, const TAcc* __restrict__ vals,
    int M1, const TIn* __restrict__ X, int ldx, int wx, const int* __restrict__ eptr,
    const int* __restrict__ eperm, const int* __restrict__ ek, const int* __restrict__ ej,
    const TAcc* __restrict__ ec, int npair, const int* __restrict__ pk, const int* __restrict__ pj,
    const int* __restrict__ epair, int pairs, int wy, const TB* Yin, int ldyin, TAcc alpha, TAcc beta, TO* Y,
    int ldy, int chunk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TAcc* Xs = reinterpret_cast<TAcc*>(smem_raw);
  TAcc* Vs = Xs + (size_t)chunk * wx;
  TAcc* Ss = Vs + (size_t)chunk * M1;   // pair sums (DIAG)
  int lcol[MAXO];
  output_columns<MAXO>(eperm, wy, lcol);
  for (int r = blockIdx.x; r < n; r += gridDim.x) {
    TAcc acc[MAXO];
#pragma unroll
    for (int i = 0; i < MAXO; ++i) acc[i] = TAcc(0);
    const int rb = rowptr[r], re = rowptr[r + 1];
    for (int cs = rb; cs < re; cs += chunk) {
      const int nzc = min(chunk, re - cs);
      __syncthreads();
      stage_chunk<TIn, TAcc>(cs, nzc, M1, colidx, vals, X, ldx, wx, Xs, Vs);
      cp_async_wait_all();
      __syncthreads();
      if (DIAG && pairs) {
        if (cs == rb)
          pair_chunk<TAcc, MAXO, true>(nzc, M1, Vs, Xs, wx, npair, pk, pj, Ss, lcol, acc);
        else
          pair_chunk<TAcc, MAXO, false>(nzc, M1, Vs, Xs, wx, npair, pk, pj, Ss, lcol, acc);
      } else if (cs == rb) {
        gather_chunk<TAcc, MAXO, DIAG, true>(nzc, M1, Vs, Xs, wx, eptr, ek, ej, ec, lcol, acc);
      } else {
        gather_chunk<TAcc, MAXO, DIAG, false>(nzc, M1, Vs, Xs, wx, eptr, ek, ej, ec, lcol, acc);
      }
    }
    if (DIAG && pairs && re > rb) {
      __syncthreads();
      pair_couple<TAcc, MAXO>(eptr, epair, ec, Ss, lcol, acc);
    }
    // Y = beta Yin + alpha sum; the two forms the solver uses (Yin - sum, and
    // the plain sum) without the multiplications (the FP64 pipe is the bound)
    const bool sub = Yin && is_value(alpha, -1.f) && is_value(beta, 1.f);
    const bool plain = !Yin && is_value(alpha, 1.f);
#pragma unroll
    for (int i = 0; i < MAXO; ++i) {
      const int l = lcol[i];
      if (l >= 0) {
        if constexpr (std::is_same_v<TAcc, df64>) {
          // double-float sums finish in FP64 (one add per output)
          const double a = acc_to_double(acc[i]);
          double v;
          if (sub) v = (double)Yin[(size_t)r * ldyin + l] - a;
          else if (plain) v = a;
          else v = df_to_scale(alpha) * a + (Yin ? df_to_scale(beta) * (double)Yin[(size_t)r * ldyin + l] : 0.0);
          Y[(size_t)r * ldy + l] = (TO)v;
        } else {
          TAcc v;
          if (sub) {
            v = (TAcc)Yin[(size_t)r * ldyin + l] - acc[i];
          } else if (plain) {
            v = acc[i];
          } else {
            v = alpha * acc[i];
            if (Yin) v += beta * (TAcc)Yin[(size_t)r * ldyin + l];
          }
          Y[(size_t)r * ldy + l] = (TO)v;
        }
      }
    }
  }
}

// Outer CG step: p_new = z + beta p_old (p_new = z on the first iteration),
// q = A p_new formed as A z + beta q_old (linearity: z is staged as it is, so
// the FP64 update is done once per output rather than once per staged
// neighbour), p_new and q written for the block's own rows, p_new . q reduced
// and alpha = rho / (p_new . q) set by the last block.
// TAcc double: FP64 arithmetic; df64: double-float products and sums on the
// FP32 units (z split exactly on staging, the values and couplings from their
// double-float copies), each output's sum finished in FP64.
template <int MAXO, int LB, typename TAcc>
__global__ void SG_MATVEC_BOUNDS(LB, MAXO) k_outer_matvec(
    int n, const int* __restrict__ rowptr, const int* __restrict__ colidx, const TAcc* __restrict__ vals,
    int M1, int P, const double* __restrict__ z, double* pA, double* pB, const int* __restrict__ eptr,
    const int* __restrict__ eperm, const int* __restrict__ ek, const int* __restrict__ ej,
    const TAcc* __restrict__ ec, int npair, const int* __restrict__ pk, const int* __restrict__ pj,
    const int* __restrict__ epair, int pairs, double* __restrict__ q, int chunk, OuterArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TAcc* Xs = reinterpret_cast<TAcc*>(smem_raw);
  TAcc* Vs = Xs + (size_t)chunk * P;
  TAcc* Ss = Vs + (size_t)chunk * M1;
  int lcol[MAXO];
  output_columns<MAXO>(eperm, P, lcol);
  const int it = a.ctl->it;
  const bool first = it == 0;
  const double beta = first ? 0.0 : a.sc[SC_BETA];
  const double* __restrict__ pold = (it & 1) ? pB : pA;
  double* __restrict__ pnew = (it & 1) ? pA : pB;
  double dot = 0.0;
  for (int r = blockIdx.x; r < n; r += gridDim.x) {
    TAcc acc[MAXO];
#pragma unroll
    for (int i = 0; i < MAXO; ++i) acc[i] = TAcc(0);
    const int rb = rowptr[r], re = rowptr[r + 1];
    for (int cs = rb; cs < re; cs += chunk) {
      const int nzc = min(chunk, re - cs);
      __syncthreads();
      stage_chunk<double, TAcc>(cs, nzc, M1, colidx, vals, z, P, P, Xs, Vs);
      cp_async_wait_all();
      __syncthreads();
      if (pairs) {
        if (cs == rb)
          pair_chunk<TAcc, MAXO, true>(nzc, M1, Vs, Xs, P, npair, pk, pj, Ss, lcol, acc);
        else
          pair_chunk<TAcc, MAXO, false>(nzc, M1, Vs, Xs, P, npair, pk, pj, Ss, lcol, acc);
      } else if (cs == rb) {
        gather_chunk<TAcc, MAXO, true, true>(nzc, M1, Vs, Xs, P, eptr, ek, ej, ec, lcol, acc);
      } else {
        gather_chunk<TAcc, MAXO, true, false>(nzc, M1, Vs, Xs, P, eptr, ek, ej, ec, lcol, acc);
      }
    }
    if (pairs && re > rb) {
      __syncthreads();
      pair_couple<TAcc, MAXO>(eptr, epair, ec, Ss, lcol, acc);
    }
#pragma unroll
    for (int i = 0; i < MAXO; ++i) {
      const int l = lcol[i];
      if (l >= 0) {
        const size_t g = (size_t)r * P + l;
        const double av = acc_to_double(acc[i]);
        const double pv = first ? z[g] : z[g] + beta * pold[g];
        const double qv = first ? av : av + beta * q[g];
        pnew[g] = pv;
        q[g] = qv;
        dot += pv * qv;
      }
    }
  }
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

// Block size of a product with wy outputs: whole warps, one output per thread
// up to 256 outputs (no idle warp and at most 31 idle lanes), 256 beyond.
static int pick_threads(int wy) { return std::min(256, 32 * std::max(1, ceil_div(wy, 32))); }

// Nonzeros staged per chunk: a whole row where 96 KB hold it, fewer for very
// wide rows. `extra` bytes (the pair sums) come on top, within the device's
// per-block limit.
static int pick_chunk(const sg_problem* h, int wx, size_t es, int M1, size_t extra, size_t* smem) {
  const size_t smem_cap = 96 * 1024;
  const size_t per_nz = (size_t)(wx + M1) * es;
  int chunk = (int)std::min<size_t>((size_t)std::max(h->max_row_nnz, 1), smem_cap / per_nz);
  const size_t limit = (size_t)std::max(h->smem_optin, 48 * 1024) - 1024;
  if (extra + (size_t)chunk * per_nz > limit) chunk = extra < limit ? (int)((limit - extra) / per_nz) : 0;
  *smem = (size_t)std::max(chunk, 1) * per_nz + extra;
  return chunk;
}

template <typename TIn, typename TAcc, typename TB, typename TO, bool DIAG>
static int launch_t(sg_problem* h, const TIn* X, int ldx, int wx, const EdgeList& E, const TB* Yin, int ldyin,
                    double alpha, double beta, TO* Y, int ldy, cudaStream_t s) {
  const int wy = E.nout;
  if (wy == 0) return SG_OK;
  const int M1 = h->nterm;
  const TAcc* vals = nullptr;
  const TAcc* ec = nullptr;
  constexpr bool DF = std::is_same_v<TAcc, df64>;
  constexpr int tk = (sizeof(TAcc) == 8 && !DF) ? SG_F64 : SG_F32;   // tuned shapes: FP64, or FP32 units
  if constexpr (DF) {
    vals = (const TAcc*)h->vals_df;
    ec = (const TAcc*)E.cdf;
  } else if constexpr (sizeof(TAcc) == 8) {
    vals = (const TAcc*)h->vals64;
    ec = (const TAcc*)E.c64;
  } else {
    vals = (const TAcc*)h->vals32;
    ec = (const TAcc*)E.c32;
  }
  int threads = pick_threads(wy);
  const int tuned = h->k1_threads[tk];
  if (DIAG && tuned > 0) threads = tuned;   // the full SG product: autotuned block size
  const int maxo = (wy + threads - 1) / threads;
  size_t smem = 0;
  const int pairs = DIAG && h->k1_pairs[tk] ? 1 : 0;
  const int chunk = pick_chunk(h, wx, sizeof(TAcc), M1, pairs ? (size_t)E.npair * sizeof(TAcc) : 0, &smem);
  if (chunk < 1) {
    set_error("block matvec: row of %d values does not fit in shared memory", wx);
    return SG_ERR_UNSUPPORTED;
  }
  auto go = [&](auto kern) -> int {
    SG_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    const int grid = std::min(h->n, h->num_sms * std::max(per_sm, 1));
    { kern<<<grid, threads, smem, s>>>(h->n, h->rowptr, h->colidx, vals, M1, X, ldx, wx, E.ptr, E.perm, E.k, E.j, ec, E.npair, E.pk, E.pj, E.pair, pairs, wy, Yin, ldyin, (TAcc)alpha, (TAcc)beta, Y, ldy, chunk); ::sghsc::note_launch(); }
    SG_CHECK_LAUNCH();
    return SG_OK;
  };
  if (threads > 256) {
    if (maxo <= 1) return go(k_block_matvec<TIn, TAcc, TB, TO, DIAG, 1, 1024>);
    if (maxo <= 2) return go(k_block_matvec<TIn, TAcc, TB, TO, DIAG, 2, 1024>);
    if (maxo <= 4) return go(k_block_matvec<TIn, TAcc, TB, TO, DIAG, 4, 1024>);
  } else {
    if (maxo <= 1) return go(k_block_matvec<TIn, TAcc, TB, TO, DIAG, 1, 256>);
    if (maxo <= 2) return go(k_block_matvec<TIn, TAcc, TB, TO, DIAG, 2, 256>);
    if (maxo <= 4) return go(k_block_matvec<TIn, TAcc, TB, TO, DIAG, 4, 256>);
    if (maxo <= 8) return go(k_block_matvec<TIn, TAcc, TB, TO, DIAG, 8, 256>);
  }
  set_error("block matvec: %d output columns exceed the supported 2048", wy);
  return SG_ERR_UNSUPPORTED;
}

int launch_block_matvec(sg_problem* h, int tin, int tacc, int tb, int tout, const void* X, int ldx, int wx,
                        const EdgeList& E, bool diag, const void* Yin, int ldyin, double alpha, double beta,
                        void* Y, int ldy, cudaStream_t s) {
  // the narrow level products: one thread per (row, output)
  const bool sub_form = !diag && Yin && alpha == -1.0 && beta == 1.0;
  if (sub_form && tin == tacc && tin == tb && tin == tout && (tin == SG_F64 || tin == SG_F32) &&
      narrow_usable(h, E, wx)) {
    if (tin == SG_F64)
      return launch_level_narrow<double>(h, E, (const double*)X, ldx, (const double*)Yin, ldyin, (double*)Y, ldy, s);
    return launch_level_narrow<float>(h, E, (const float*)X, ldx, (const float*)Yin, ldyin, (float*)Y, ldy, s);
  }
  if (tin == SG_F64 && tacc == SG_F64 && tb == SG_F64 && tout == SG_F64) {
    auto Xp = (const double*)X;
    auto Bp = (const double*)Yin;
    auto Yp = (double*)Y;
    if (diag) return launch_t<double, double, double, double, true>(h, Xp, ldx, wx, E, Bp, ldyin, alpha, beta, Yp, ldy, s);
    return launch_t<double, double, double, double, false>(h, Xp, ldx, wx, E, Bp, ldyin, alpha, beta, Yp, ldy, s);
  }
  if (tin == SG_F32 && tacc == SG_F32 && tb == SG_F32 && tout == SG_F32) {
    auto Xp = (const float*)X;
    auto Bp = (const float*)Yin;
    auto Yp = (float*)Y;
    // the row kernel with input columns in registers for the full product and the wide level products
    const bool plain = diag && !Yin && alpha == 1.0 && beta == 0.0;
    const bool sub = !diag && Yin && alpha == -1.0 && beta == 1.0;
    if ((plain || sub) && rows32_usable(h, E, wx, diag))
      return launch_rows32(h, E, diag, Xp, ldx, wx, Bp, ldyin, Yp, ldy, s);
    if (diag) return launch_t<float, float, float, float, true>(h, Xp, ldx, wx, E, Bp, ldyin, alpha, beta, Yp, ldy, s);
    return launch_t<float, float, float, float, false>(h, Xp, ldx, wx, E, Bp, ldyin, alpha, beta, Yp, ldy, s);
  }
  if (tin == SG_F32 && tacc == SG_F64 && tb == SG_F64 && tout == SG_F32 && !diag) {
    return launch_t<float, double, double, float, false>(h, (const float*)X, ldx, wx, E, (const double*)Yin, ldyin,
                                                         alpha, beta, (float*)Y, ldy, s);
  }
  if (tin == SG_F32 && tacc == ACC_DF64 && tout == SG_F64 && diag && !Yin) {
    if (alpha == 1.0 && df_pairs_usable(h, E, wx) && &E == &h->all && wx == h->P && ldx == h->P && ldy == h->P)
      return launch_df_apply(h, (const float*)X, (double*)Y, s);
    return launch_t<float, df64, double, double, true>(h, (const float*)X, ldx, wx, E, nullptr, 0, alpha, beta,
                                                       (double*)Y, ldy, s);
  }
  if (tin == SG_F32 && tacc == ACC_DF64 && tb == SG_F64 && tout == SG_F32 && !diag) {
    if (Yin && alpha == -1.0 && beta == 1.0 && df_pairs_usable(h, E, wx))
      return launch_df_level(h, E, (const float*)X, ldx, wx, (const double*)Yin, ldyin, (float*)Y, ldy, s);
    return launch_t<float, df64, double, float, false>(h, (const float*)X, ldx, wx, E, (const double*)Yin, ldyin,
                                                       alpha, beta, (float*)Y, ldy, s);
  }
  set_error("block matvec: unsupported type combination");
  return SG_ERR_UNSUPPORTED;
}

template <typename TAcc>
static int launch_outer_t(sg_problem* h, const OuterArgs& a, cudaStream_t s) {
  constexpr bool DF = std::is_same_v<TAcc, df64>;
  const int P = h->P, M1 = h->nterm;
  // whole warps, <= 1024: the autotuned block size or 256 (the double-float
  // form has its own tuned shape)
  const int tuned = DF ? h->outer_threads_df : h->outer_threads;
  const int threads = tuned > 0 ? tuned : 256;
  const int maxo = (P + threads - 1) / threads;
  size_t smem = 0;
  const int pairs = (DF ? h->outer_pairs_df : h->outer_pairs) ? 1 : 0;
  const int chunk = pick_chunk(h, P, sizeof(TAcc), M1, pairs ? (size_t)h->all.npair * sizeof(TAcc) : 0, &smem);
  if (chunk < 1) {
    set_error("outer matvec: P = %d does not fit in shared memory", P);
    return SG_ERR_UNSUPPORTED;
  }
  const TAcc* vals = DF ? (const TAcc*)h->vals_df : (const TAcc*)h->vals64;
  const TAcc* ec = DF ? (const TAcc*)h->all.cdf : (const TAcc*)h->all.c64;
  auto go = [&](auto kern) -> int {
    SG_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    const int grid = std::min(std::min(h->n, h->num_sms * std::max(per_sm, 1)), h->opart_blocks);
    { kern<<<grid, threads, smem, s>>>(h->n, h->rowptr, h->colidx, vals, M1, P, h->fz, h->fpA, h->fpB, h->all.ptr, h->all.perm, h->all.k, h->all.j, ec, h->all.npair, h->all.pk, h->all.pj, h->all.pair, pairs, h->fq, chunk, a); ::sghsc::note_launch(); }
    SG_CHECK_LAUNCH();
    return SG_OK;
  };
  if (threads > 256) {
    if (maxo <= 1) return go(k_outer_matvec<1, 1024, TAcc>);
    if (maxo <= 2) return go(k_outer_matvec<2, 1024, TAcc>);
    if (maxo <= 4) return go(k_outer_matvec<4, 1024, TAcc>);
  } else {
    if (maxo <= 1) return go(k_outer_matvec<1, 256, TAcc>);
    if (maxo <= 2) return go(k_outer_matvec<2, 256, TAcc>);
    if (maxo <= 4) return go(k_outer_matvec<4, 256, TAcc>);
    if (maxo <= 8) return go(k_outer_matvec<8, 256, TAcc>);
  }
  set_error("outer matvec: P = %d exceeds the supported 2048", P);
  return SG_ERR_UNSUPPORTED;
}

int launch_outer_matvec(sg_problem* h, const OuterArgs& a, cudaStream_t s, bool df, const float* z32) {
  if (df && df_pairs_usable(h, h->all, h->P)) return launch_df_outer(h, a, s, z32);
  return df ? launch_outer_t<df64>(h, a, s) : launch_outer_t<double>(h, a, s);
}

}  // namespace sghsc

using namespace sghsc;

extern "C" {

int sg_apply(sg_problem* h, const void* U, void* Y, int dtype, void* stream) {
  set_error("");
  if (!h || !U || !Y || (dtype != SG_F64 && dtype != SG_F32 && dtype != SG_F32_ACCDF64) || U == Y) {
    set_error("sg_apply: invalid arguments");
    return SG_ERR_INVALID_ARG;
  }
  if (dtype == SG_F32_ACCDF64)   // FP32 U, FP64-accurate sums, FP64 Y
    return launch_block_matvec(h, SG_F32, ACC_DF64, SG_F64, SG_F64, U, h->P, h->P, h->all, true, nullptr, 0, 1.0, 0.0,
                               Y, h->P, (cudaStream_t)stream);
  return launch_block_matvec(h, dtype, dtype, dtype, dtype, U, h->P, h->P, h->all, true, nullptr, 0, 1.0, 0.0, Y,
                             h->P, (cudaStream_t)stream);
}

int sg_level_apply(sg_problem* h, int lvl_out, int lvl_in, const void* X, const void* Yin, void* Yout, int dtype,
                   void* stream) {
  set_error("");
  const bool mixed = dtype == SG_F32_ACC64 || dtype == SG_F32_ACCDF64;
  if (!h || !X || !Yout || (dtype != SG_F64 && dtype != SG_F32 && !mixed) || lvl_out < 0 || lvl_in < 0 ||
      lvl_out > h->p || lvl_in > h->p || (lvl_out - lvl_in != 1 && lvl_in - lvl_out != 1) ||
      (mixed && (!Yin || Yin == (const void*)Yout))) {
    set_error("sg_level_apply: invalid arguments");
    return SG_ERR_INVALID_ARG;
  }
  const EdgeList& E = lvl_in > lvl_out ? h->pre[lvl_in] : h->post[lvl_out];
  const int win = h->off[lvl_in + 1] - h->off[lvl_in];
  const int wout = h->off[lvl_out + 1] - h->off[lvl_out];
  if (mixed)   // the level-p products of the mixed preconditioner with an FP64-accurate top level
    return launch_block_matvec(h, SG_F32, dtype == SG_F32_ACC64 ? SG_F64 : ACC_DF64, SG_F64, SG_F32, X, win, win, E,
                               false, Yin, wout, -1.0, 1.0, Yout, wout, (cudaStream_t)stream);
  return launch_block_matvec(h, dtype, dtype, dtype, dtype, X, win, win, E, false, Yin, wout, -1.0, 1.0, Yout, wout,
                             (cudaStream_t)stream);
}

}  // extern "C"
