// K7: the quantity of interest Q = E[int u^2] = sum_j u_j^T M_h u_j and the
// adjoint gradient contraction h_k = <Lam, A_k U G_k^T>_F (k = 0..M), fused
// into one pass over the shared CSR pattern: the K1 gather with a reduction
// epilogue instead of a store. The paper has no gradient; the operator is
// symmetric (Sec. 3, the symmetry remark), so the adjoint solve is one more
// preconditioned solve with the same operator and dQ/dtheta =
// -sum_k (d A_k / d theta) contracted as above.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sghsc_internal.cuh"
#include "vec.cuh"

namespace sghsc {

constexpr int QOI_MAXK = 32;

// dQdU = 2 M_h U (optional), per-block partials of sum U .* (M_h U)
__global__ void __launch_bounds__(256) k_mass(int n, int P, const int* __restrict__ rowptr,
                                              const int* __restrict__ colidx, const double* __restrict__ mass,
                                              const double* __restrict__ U, double* __restrict__ dQdU,
                                              double* __restrict__ part) {
  double acc = 0.0;
  for (int r = blockIdx.x; r < n; r += gridDim.x) {
    const int rb = rowptr[r], re = rowptr[r + 1];
    for (int l = threadIdx.x; l < P; l += blockDim.x) {
      double s = 0.0;
      for (int e = rb; e < re; ++e) s += mass[e] * U[(size_t)colidx[e] * P + l];
      if (dQdU) dQdU[(size_t)r * P + l] = 2.0 * s;
      acc += U[(size_t)r * P + l] * s;
    }
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Per-block partials part[b][k] of h_k = sum_{r,l} Lam(r,l) (A_k U G_k^T)(r,l).
__global__ void __launch_bounds__(256) k_grad(int n, int P, int M1, const int* __restrict__ rowptr,
                                              const int* __restrict__ colidx, const double* __restrict__ vals,
                                              const double* __restrict__ U, const double* __restrict__ Lam,
                                              const int* __restrict__ eptr, const int* __restrict__ ek,
                                              const int* __restrict__ ej, const double* __restrict__ ec,
                                              int chunk, double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* Xs = reinterpret_cast<double*>(smem_raw);
  double* Vs = Xs + (size_t)chunk * P;
  double hk[QOI_MAXK];
  for (int k = 0; k < M1; ++k) hk[k] = 0.0;
  for (int r = blockIdx.x; r < n; r += gridDim.x) {
    const int rb = rowptr[r], re = rowptr[r + 1];
    for (int cs = rb; cs < re; cs += chunk) {
      const int nzc = min(chunk, re - cs);
      __syncthreads();
      for (int idx = threadIdx.x; idx < nzc * P; idx += blockDim.x) {
        const int e = idx / P, j = idx - e * P;
        cp_async_elem(Xs + idx, U + (size_t)colidx[cs + e] * P + j);
      }
      for (int idx = threadIdx.x; idx < nzc * M1; idx += blockDim.x) cp_async_elem(Vs + idx, vals + (size_t)cs * M1 + idx);
      cp_async_wait_all();
      __syncthreads();
      for (int l = threadIdx.x; l < P; l += blockDim.x) {
        const double lam = Lam[(size_t)r * P + l];
        double a0 = 0.0;
        for (int e = 0; e < nzc; ++e) a0 += Vs[e * M1] * Xs[e * P + l];
        hk[0] += lam * a0;
        for (int t = eptr[l]; t < eptr[l + 1]; ++t) {
          const int k = ek[t], j = ej[t];
          double s = 0.0;
          for (int e = 0; e < nzc; ++e) s += Vs[e * M1 + k] * Xs[e * P + j];
          hk[k] += lam * ec[t] * s;
        }
      }
    }
  }
  __shared__ double red[256];
  for (int k = 0; k < M1; ++k) {
    __syncthreads();
    red[threadIdx.x] = hk[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * M1 + k] = red[0];
  }
}

// grad[t] = sum_k W[t][k] h_k with h_k the fixed-order sum of the partials.
__global__ void k_grad_fin(int nblk, int M1, int nparam, const double* __restrict__ part,
                           const double* __restrict__ W, double* __restrict__ grad, double* __restrict__ hk_out) {
  __shared__ double hk[QOI_MAXK];
  if ((int)threadIdx.x < M1) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)b * M1 + threadIdx.x];
    hk[threadIdx.x] = s;
    if (hk_out) hk_out[threadIdx.x] = s;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nparam; t += blockDim.x) {
    double g = 0.0;
    for (int k = 0; k < M1; ++k) g += W[(size_t)t * M1 + k] * hk[k];
    grad[t] = g;
  }
}

__global__ void k_sum_fin(int nblk, const double* __restrict__ part, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[b];
    *out = s;
  }
}

static int ensure_part(sg_problem* h, size_t count) {
  if (h->opart && (size_t)h->opart_blocks * 2 >= count) return SG_OK;
  clear_graphs(h);   // captured solve graphs use the partial-sum buffer
  SG_TRY_CUDA(cudaDeviceSynchronize());
  cudaFree(h->opart);
  h->opart = nullptr;
  h->opart_blocks = 0;
  const int blocks = (int)std::max<size_t>((count + 1) / 2, (size_t)h->num_sms * 16);
  SG_TRY_CUDA(cudaMalloc((void**)&h->opart, (size_t)blocks * 2 * sizeof(double)));
  h->opart_blocks = blocks;
  return SG_OK;
}

// The gradient workload's parameters theta = (a_mean, sigma, s_1..s_M) act on
// matrices given to sg_setup with unit parameters (A_0 = L_h, A_k = Phi_k):
// A_0(theta) = a_mean L_h and A_k(theta) = sigma s_k Phi_k. scale[k] is the
// factor of A_k; W[t][k] = -d log(scale[k]) / d theta_t turns the contractions
// h_k = <Lam, A_k U G_k^T> into dQ/dtheta_t = sum_k W[t][k] h_k (the adjoint
// formula dQ/dtheta = -Lam^T (dA/dtheta) U with dA_k/dtheta_t = A_k d log
// scale[k] / d theta_t).
static int theta_check(const sg_problem* h, const double* theta, const char* name) {
  if (!h || !theta) {
    set_error("%s: invalid arguments", name);
    return SG_ERR_INVALID_ARG;
  }
  if (h->q >= 0) {
    set_error("%s: the parameterisation is that of the linear KL expansion", name);
    return SG_ERR_UNSUPPORTED;
  }
  for (int t = 0; t < h->M + 2; ++t)
    if (!std::isfinite(theta[t]) || theta[t] == 0.0) {
      set_error("%s: theta[%d] must be finite and nonzero", name, t);
      return SG_ERR_INVALID_ARG;
    }
  if (!(theta[0] > 0.0)) {
    set_error("%s: a_mean = theta[0] must be positive", name);
    return SG_ERR_INVALID_ARG;
  }
  return SG_OK;
}

static void theta_scales(int M, const double* theta, std::vector<double>& scale) {
  scale.assign(M + 1, 0.0);
  scale[0] = theta[0];
  for (int k = 1; k <= M; ++k) scale[k] = theta[1] * theta[1 + k];
}

static void theta_weights(int M, const double* theta, std::vector<double>& W) {
  const int M1 = M + 1;
  W.assign((size_t)(M + 2) * M1, 0.0);
  W[0] = -1.0 / theta[0];
  for (int k = 1; k <= M; ++k) {
    W[(size_t)1 * M1 + k] = -1.0 / theta[1];
    W[(size_t)(1 + k) * M1 + k] = -1.0 / theta[1 + k];
  }
}

}  // namespace sghsc

using namespace sghsc;

extern "C" {

int sg_qoi(sg_problem* h, const double* U, double* dQdU, double* q_out, void* stream) {
  set_error("");
  if (!h || !U || !q_out || !h->mass64) {
    set_error("sg_qoi: invalid arguments or no mass matrix given to sg_setup");
    return SG_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = std::min(h->n, h->num_sms * 8);
  SG_TRY(ensure_part(h, grid));
  { k_mass<<<grid, 256, 0, s>>>(h->n, h->P, h->rowptr, h->colidx, h->mass64, U, dQdU, h->opart); ::sghsc::note_launch(); }
  { k_sum_fin<<<1, 32, 0, s>>>(grid, h->opart, q_out); ::sghsc::note_launch(); }
  SG_CHECK_LAUNCH();
  return SG_OK;
}

int sg_qoi_grad(sg_problem* h, const double* U, const double* Lam, int nparam, const double* W, double* grad,
                double* hk_out, void* stream) {
  set_error("");
  const int M1 = h ? h->nterm : 0;
  if (!h || !U || !Lam || !W || !grad || nparam < 1 || M1 > QOI_MAXK) {
    set_error("sg_qoi_grad: invalid arguments (the value terms, M+1, must be <= %d)", QOI_MAXK);
    return SG_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t wcount = (size_t)nparam * M1;
  if ((size_t)h->wdev_cap < wcount) {
    cudaFree(h->wdev);
    h->wdev = nullptr;
    h->wdev_cap = 0;
    SG_TRY_CUDA(cudaMalloc((void**)&h->wdev, wcount * sizeof(double)));
    h->wdev_cap = (int)wcount;
  }
  SG_TRY_CUDA(cudaMemcpyAsync(h->wdev, W, wcount * sizeof(double), cudaMemcpyHostToDevice, s));
  const size_t per_nz = (size_t)(h->P + M1) * sizeof(double);
  const int chunk = (int)std::min<size_t>((size_t)std::max(h->max_row_nnz, 1), (96 * 1024) / per_nz);
  if (chunk < 1) {
    set_error("sg_qoi_grad: P too large for shared memory");
    return SG_ERR_UNSUPPORTED;
  }
  const size_t smem = (size_t)chunk * per_nz;
  SG_TRY_CUDA(cudaFuncSetAttribute(k_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 1;
  SG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grad, 256, smem));
  const int grid = std::min(h->n, h->num_sms * std::max(per_sm, 1));
  SG_TRY(ensure_part(h, (size_t)grid * M1));
  { k_grad<<<grid, 256, smem, s>>>(h->n, h->P, M1, h->rowptr, h->colidx, h->vals64, U, Lam, h->all.ptr, h->all.k,
                                 h->all.j, h->all.c64, chunk, h->opart); ::sghsc::note_launch(); }
  { k_grad_fin<<<1, 64, 0, s>>>(grid, M1, nparam, h->opart, h->wdev, grad, hk_out); ::sghsc::note_launch(); }
  SG_CHECK_LAUNCH();
  // W is a host buffer: keep it alive until the copy above has run
  SG_TRY_CUDA(cudaStreamSynchronize(s));
  return SG_OK;
}

int sg_kl_set_theta(sg_problem* h, const double* theta) {
  set_error("");
  SG_TRY(theta_check(h, theta, "sg_kl_set_theta"));
  std::vector<double> scale;
  theta_scales(h->M, theta, scale);
  return sg_set_scales(h, scale.data());
}

int sg_kl_qoi_grad(sg_problem* h, const double* U, const double* Lam, const double* theta, double* grad,
                   double* hk_out, void* stream) {
  set_error("");
  SG_TRY(theta_check(h, theta, "sg_kl_qoi_grad"));
  std::vector<double> W;
  theta_weights(h->M, theta, W);
  return sg_qoi_grad(h, U, Lam, h->M + 2, W.data(), grad, hk_out, stream);
}

}  // extern "C"
