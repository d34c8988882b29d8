// FP32 SG products (eq. (3): Y = sum_k A_k X G_k^T, the full product or a
// level product B_l / C_l of Algorithm 1) with every input column in
// registers.
//
// One block per matrix row r at a time (two on narrower levels). For each chunk of up to nine
// nonzeros c_e of the row (the Q1 stencil row is one chunk) the block stages
// the KL-term values a_k(r, c_e) in shared memory, padded to three float4 per
// term; thread j then loads X(c_e, j) for its input column from global memory
// (coalesced across the warp, L2-resident across the nine rows that share a
// neighbour) and forms the stencil sums T(k, j) = sum_e a_k(r, c_e) X(c_e, j)
// for every term k, reading the term's values as broadcast float4: three
// shared loads per nine FMAs. T (M+1 x wx, FP32) is the only large shared
// array. Then output l sums its couplings c * T(k, j) (and T(0, l) for the
// identity of G_0 in the full product) from a slot-transposed table of
// packed (class, offset of T(k, j)) words read coalesced through L1, and
// writes Y(r, l) or Yin(r, l) - that.
//
// T is formed for every (k, j) although the couplings use about half of them
// at M = 10, p = 4: the extra FMAs cost less than the per-pair bookkeeping
// they replace (the staged pair kernel reads two shared operands per FMA).
#include <cuda_runtime.h>

#include "sghsc_internal.cuh"
#include "vec.cuh"

namespace sghsc {

namespace rows32 {
constexpr int NT = ROWS32_COLS / 2;   // threads per block
constexpr int CH = 9;     // nonzeros per chunk
constexpr int VS4 = 3;    // float4 per term row of the staged values (12 slots)
}  // namespace rows32

// sum_e a(e) x(e) over the nine slots of one term row (three float4, the
// last three slots unused), for two input columns
__device__ __forceinline__ void term_sum2(const float4* v, const float (&x)[rows32::CH],
                                          const float (&y)[rows32::CH], float& sx, float& sy) {
  const float4 a = v[0], b = v[1];
  const float c = v[2].x;
  sx = a.x * x[0];
  sy = a.x * y[0];
  sx = fmaf(a.y, x[1], sx);
  sy = fmaf(a.y, y[1], sy);
  sx = fmaf(a.z, x[2], sx);
  sy = fmaf(a.z, y[2], sy);
  sx = fmaf(a.w, x[3], sx);
  sy = fmaf(a.w, y[3], sy);
  sx = fmaf(b.x, x[4], sx);
  sy = fmaf(b.x, y[4], sy);
  sx = fmaf(b.y, x[5], sx);
  sy = fmaf(b.y, y[5], sy);
  sx = fmaf(b.z, x[6], sx);
  sy = fmaf(b.z, y[6], sy);
  sx = fmaf(b.w, x[7], sx);
  sy = fmaf(b.w, y[7], sy);
  sx = fmaf(c, x[8], sx);
  sy = fmaf(c, y[8], sy);
}


// DIAG: add T(0, l) (full product); SUB: Y = Yin - sum (Yin may alias Y:
// each entry is read, then written, by the same thread), else Y = sum.
// ROWS rows at a time, RG = NT / ROWS threads per row (a multiple of 32, so
// the slot-transposed couplings still give a warp consecutive words): on
// narrow levels several rows share the block's barriers.
template <bool DIAG, bool SUB, int ROWS>
__global__ void __launch_bounds__(rows32::NT, 4) k_rows32(
    int n, const int* __restrict__ rowptr, const int* __restrict__ colidx, const float* __restrict__ vals, int M1,
    const float* __restrict__ X, int ldx, int wx, const unsigned* __restrict__ ckj, const int2* __restrict__ sdesc,
    const float* __restrict__ ctab, int ncls, int wy, const float* Yin, int ldyin, float* Y, int ldy) {
  using namespace rows32;
  constexpr int RG = NT / ROWS;
  extern __shared__ __align__(16) float4 sm4[];
  const int wts = rows32_stride(wx);
  float* Ctab = reinterpret_cast<float*>(sm4);                        // [ncls]
  float4* Vall = sm4 + (ncls + 3) / 4;                                 // [ROWS][M1][VS4]
  float* Tall = reinterpret_cast<float*>(Vall + (size_t)ROWS * M1 * VS4);   // [ROWS][M1][wts]
  const int tid = threadIdx.x, g = tid / RG, lt = tid - g * RG;
  float4* Vt = Vall + (size_t)g * M1 * VS4;
  float* Vf = reinterpret_cast<float*>(Vt);
  float* Ts = Tall + (size_t)g * M1 * wts;
  for (int t = tid; t < ncls; t += NT) Ctab[t] = ctab[t];
  for (long long rbase = (long long)blockIdx.x * ROWS; rbase < n; rbase += (long long)gridDim.x * ROWS) {
    const int r = (int)rbase + g;
    const bool rv = r < n;
    const int rb = rv ? rowptr[r] : 0, re = rv ? rowptr[r + 1] : 0;
    int maxnz = re - rb;   // chunks of the block's longest row: every thread runs the same barriers
#pragma unroll
    for (int q = 0; q < ROWS; ++q) {
      const long long rq = rbase + q;
      if (ROWS > 1 && rq < n) maxnz = max(maxnz, rowptr[rq + 1] - rowptr[rq]);
    }
    for (int cs = 0; cs < maxnz; cs += CH) {
      const int nzc = max(0, min(CH, re - rb - cs));
      __syncthreads();   // Vt (previous chunk) and T (previous rows' couplings) are read no more
      for (int t = lt; t < M1 * VS4 * 4; t += RG) {
        const int k = t / (VS4 * 4), e = t - k * (VS4 * 4);
        Vf[t] = e < nzc ? vals[(size_t)(rb + cs + e) * M1 + k] : 0.f;
      }
      int col[CH];
#pragma unroll
      for (int e = 0; e < CH; ++e) col[e] = e < nzc ? colidx[rb + cs + e] : -1;
      __syncthreads();
      const bool first = cs == 0;
      // two input columns per thread (j0, j0 + RG): each staged term row feeds
      // 18 FMAs; columns past wx read nothing and fill the padding of T
      for (int j0 = lt; j0 < wx; j0 += 2 * RG) {
        const int j1 = j0 + RG;
        float x0[CH], x1[CH];
#pragma unroll
        for (int e = 0; e < CH; ++e) {
          x0[e] = col[e] >= 0 ? X[(size_t)col[e] * ldx + j0] : 0.f;
          x1[e] = (col[e] >= 0 && j1 < wx) ? X[(size_t)col[e] * ldx + j1] : 0.f;
        }
        float* tp = Ts + j0;
        if (first) {
#pragma unroll 2
          for (int k = 0; k < M1; ++k, tp += wts) {
            float s0, s1;
            term_sum2(Vt + k * VS4, x0, x1, s0, s1);
            tp[0] = s0;
            tp[RG] = s1;
          }
        } else {
#pragma unroll 2
          for (int k = 0; k < M1; ++k, tp += wts) {
            float s0, s1;
            term_sum2(Vt + k * VS4, x0, x1, s0, s1);
            tp[0] += s0;
            tp[RG] += s1;
          }
        }
      }
    }
    __syncthreads();
    if (!rv) continue;
    // outputs by slot (sorted by coupling count, so a warp's loops end together)
    for (int slot = lt; slot < wy; slot += RG) {
      const int2 d = __ldg(sdesc + slot);
      const int l = (int)((unsigned)d.y >> 16), ncl = d.y & 0xffff;
      float acc = 0.f;
      if (re > rb) {
        if (DIAG) acc = Ts[l];
        const unsigned* cw = ckj + d.x;
        int c = 0;
        for (; c + 4 <= ncl; c += 4, cw += 128) {
          const unsigned w0 = __ldg(cw), w1 = __ldg(cw + 32), w2 = __ldg(cw + 64), w3 = __ldg(cw + 96);
          acc = fmaf(Ctab[w0 >> 24], Ts[w0 & 0xffffffu], acc);
          acc = fmaf(Ctab[w1 >> 24], Ts[w1 & 0xffffffu], acc);
          acc = fmaf(Ctab[w2 >> 24], Ts[w2 & 0xffffffu], acc);
          acc = fmaf(Ctab[w3 >> 24], Ts[w3 & 0xffffffu], acc);
        }
        for (; c < ncl; ++c, cw += 32) {
          const unsigned w = __ldg(cw);
          acc = fmaf(Ctab[w >> 24], Ts[w & 0xffffffu], acc);
        }
      }
      if (SUB) Y[(size_t)r * ldy + l] = Yin[(size_t)r * ldyin + l] - acc;
      else Y[(size_t)r * ldy + l] = acc;
    }
  }
}

static size_t rows32_smem(const EdgeList& E, int M1, int wx, int rows) {
  return (size_t)((E.ncls + 3) & ~3) * 4 +
         (size_t)rows * ((size_t)M1 * rows32::VS4 * 16 + (size_t)M1 * rows32_stride(wx) * 4);
}

// Rows per block: one for the wide products, two for the level products
// between 32 and 512 columns each way (at 511^2 rows, M = 10: 55 <- 220
// columns 0.95 against 1.36 ms for the row-per-warp kernel, 220 <- 55 0.90
// against 0.98 ms; four rows per block: 1.10 and 1.12 ms); 0 where this
// kernel is not taken.
static int rows32_rows(const EdgeList& E, int wx, bool diag) {
  if (wx >= 512 || E.nout >= 512) return 1;
  return !diag && wx >= 32 && E.nout >= 32 ? 2 : 0;
}

// FP32 products take this kernel for inputs from 512 columns, or from 128
// input columns with at least 512 outputs (measured on the 512x512, M = 10,
// p = 4 operator: 1001 -> 1001 columns 3.7 ms against 11.1 ms for the
// row-per-warp kernel, 715 -> 220 2.7 against 4.6 ms, 220 -> 715 2.0 against
// 3.4 ms), and with two rows per block for level products of 32 to 512
// columns each way (one row per block there: 220 -> 55 1.16 against
// 0.99 ms, the rows too short to amortise the block barriers).
bool rows32_usable(const sg_problem* h, const EdgeList& E, int wx, bool diag) {
  const int rows = rows32_rows(E, wx, diag);
  const bool shape = wx >= 512 || (E.nout >= 512 && wx >= 128) || rows > 1;
  return h->staged_pairs && shape && wx == E.nin && E.ckj && E.sdesc && E.ncls > 0 && h->nterm <= 256 &&
         rows32_smem(E, h->nterm, wx, std::max(rows, 1)) <= (size_t)std::max(h->smem_optin, 48 * 1024);
}

int launch_rows32(sg_problem* h, const EdgeList& E, bool diag, const float* X, int ldx, int wx, const float* Yin,
                  int ldyin, float* Y, int ldy, cudaStream_t s) {
  using namespace rows32;
  const int wy = E.nout;
  if (wy == 0) return SG_OK;
  if (diag == (Yin != nullptr)) {
    set_error("FP32 row product: unsupported form");
    return SG_ERR_UNSUPPORTED;
  }
  const int rows = std::max(rows32_rows(E, wx, diag), 1);
  const size_t smem = rows32_smem(E, h->nterm, wx, rows);
  auto go = [&](auto kern) -> int {
    SG_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
    const int grid = std::min((h->n + rows - 1) / rows, h->num_sms * std::max(per_sm, 1));
    { kern<<<grid, NT, smem, s>>>(h->n, h->rowptr, h->colidx, h->vals32, h->nterm, X, ldx, wx, E.ckj, E.sdesc,
                                  E.ctab32, E.ncls, wy, Yin, ldyin, Y, ldy); ::sghsc::note_launch(); }
    SG_CHECK_LAUNCH();
    return SG_OK;
  };
  if (diag) return go(k_rows32<true, false, 1>);
  if (rows == 2) return go(k_rows32<false, true, 2>);
  return go(k_rows32<false, true, 1>);
}

}  // namespace sghsc
