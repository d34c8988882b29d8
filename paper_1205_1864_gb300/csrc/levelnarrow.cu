// Narrow level products of Algorithm 1 (eq. (global-matrix-hierarchy)):
// Y = Yin - sum_k A_k X G_k[out, in]^T into at most 16 output columns (B_1,
// C_1, B_2 at M = 10, p = 4: 1, 10 and 10 columns).
//
// One thread per (spatial row, output column), in the gather form: for each
// coupling (k, j, c) of output l, s = sum_e a_k(r, c_e) X(c_e, j) over the
// row's nonzeros, and the output adds c s. No shared memory and no block
// barrier: a block holds 256 / w_out' rows (w_out' = w_out rounded up to a
// power of two), every thread runs independently, and the row's values and
// the neighbour rows of X come through L1. On these widths the kernel that
// stages a row per block spends its time waiting on the row's chain of loads
// and barriers: at 511^2 rows, M = 10, 1 <- 10 columns 0.12 against 0.38 ms,
// 10 <- 1 0.06 against 0.13 ms, 10 <- 55 0.33 against 0.52 ms. From 55
// outputs on, the two loads per multiply-add through L1 cost more than the
// staging saves (55 <- 10 0.29 against 0.26 ms, 220 <- 55 1.63 against
// 0.99 ms), so wider products keep the staged kernels.
#include <cuda_runtime.h>

#include "sghsc_internal.cuh"
#include "vec.cuh"

namespace sghsc {

namespace narrow {
constexpr int NT = 256;
constexpr int MAX_OUT = 16;
}  // namespace narrow

template <typename T>
__global__ void __launch_bounds__(narrow::NT) k_level_narrow(
    int n, const int* __restrict__ rowptr, const int* __restrict__ colidx, const T* __restrict__ vals, int M1,
    const T* __restrict__ X, int ldx, const int* __restrict__ eptr, const int* __restrict__ ek,
    const int* __restrict__ ej, const T* __restrict__ ec, int wy, int wyp, const T* Yin, int ldyin, T* Y, int ldy) {
  const int rpb = narrow::NT / wyp;   // rows per block
  const int l = threadIdx.x % wyp, dr = threadIdx.x / wyp;
  if (l >= wy) return;   // no barrier below
  const int t0 = eptr[l], t1 = eptr[l + 1];
  for (long long rr = (long long)blockIdx.x * rpb + dr; rr < n; rr += (long long)gridDim.x * rpb) {
    const int r = (int)rr;
    const int rb = rowptr[r], re = rowptr[r + 1];
    T acc = T(0);
    for (int t = t0; t < t1; ++t) {
      const int k = ek[t], j = ej[t];
      T s = T(0);
      for (int q = rb; q < re; ++q) s = fma(vals[(size_t)q * M1 + k], X[(size_t)colidx[q] * ldx + j], s);
      acc = fma(ec[t], s, acc);
    }
    Y[(size_t)r * ldy + l] = Yin[(size_t)r * ldyin + l] - acc;
  }
}

bool narrow_usable(const sg_problem* h, const EdgeList& E, int wx) {
  return h->staged_pairs && E.nout > 0 && E.nout <= narrow::MAX_OUT && wx < 512 && wx == E.nin;
}

template <typename T>
int launch_level_narrow(sg_problem* h, const EdgeList& E, const T* X, int ldx, const T* Yin, int ldyin, T* Y, int ldy,
                        cudaStream_t s) {
  using namespace narrow;
  const int wy = E.nout;
  int wyp = 1;
  while (wyp < wy) wyp *= 2;
  const int rpb = NT / wyp;
  auto kern = k_level_narrow<T>;
  int per_sm = 0;
  SG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, 0));
  const long long blocks = ((long long)h->n + rpb - 1) / rpb;
  const int grid = (int)std::max(1LL, std::min(blocks, (long long)h->num_sms * std::max(per_sm, 1)));
  const T* vals = std::is_same_v<T, double> ? (const T*)h->vals64 : (const T*)h->vals32;
  const T* ec = std::is_same_v<T, double> ? (const T*)E.c64 : (const T*)E.c32;
  { kern<<<grid, NT, 0, s>>>(h->n, h->rowptr, h->colidx, vals, h->nterm, X, ldx, E.ptr, E.k, E.j, ec, wy, wyp, Yin,
                             ldyin, Y, ldy); ::sghsc::note_launch(); }
  SG_CHECK_LAUNCH();
  return SG_OK;
}

template int launch_level_narrow<float>(sg_problem*, const EdgeList&, const float*, int, const float*, int, float*,
                                        int, cudaStream_t);
template int launch_level_narrow<double>(sg_problem*, const EdgeList&, const double*, int, const double*, int,
                                         double*, int, cudaStream_t);

}  // namespace sghsc
