// ALU throughput probe: the FP64 and FP32 multiply-add rates of the device,
// measured with CUDA events on one launch of a kernel that does nothing but
// independent fused multiply-add chains. They are the roofline denominators of
// the ALU-bound kernels (the FP64 SG products), taken on the device that runs
// them instead of from unit counts and clocks. No device setting is changed.
#include <algorithm>

#include "sghsc_internal.cuh"

namespace sghsc {

// CHAINS independent chains per thread, each a <- a * m + c for `iters`
// iterations (m slightly below 1, so the values stay finite); the result is
// stored only when `sink` is set, which the host never does, but the compiler
// cannot drop the chains.
template <typename T, int CHAINS>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, T m, T c, T* sink, int store) {
  T a[CHAINS];
#pragma unroll
  for (int i = 0; i < CHAINS; ++i) a[i] = T(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
#pragma unroll
      for (int i = 0; i < CHAINS; ++i) a[i] = fma(a[i], m, c);
    }
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < CHAINS; ++i) s += a[i];
  if (store) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static int run_probe(int iters, double* flops_per_s, cudaStream_t s) {
  constexpr int CHAINS = 8;
  int dev = 0, sms = 0, per_sm = 0;
  SG_TRY_CUDA(cudaGetDevice(&dev));
  SG_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SG_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe<T, CHAINS>, 256, 0));
  const int grid = sms * std::max(per_sm, 1);
  cudaEvent_t e0, e1;
  SG_TRY_CUDA(cudaEventCreate(&e0));
  SG_TRY_CUDA(cudaEventCreate(&e1));
  // warm-up launch, then the timed one
  { k_fma_probe<T, CHAINS><<<grid, 256, 0, s>>>(std::max(iters / 8, 1), T(0.999999), T(1e-3), nullptr, 0); note_launch(); }
  cudaEventRecord(e0, s);
  { k_fma_probe<T, CHAINS><<<grid, 256, 0, s>>>(iters, T(0.999999), T(1e-3), nullptr, 0); note_launch(); }
  cudaEventRecord(e1, s);
  const cudaError_t le = cudaGetLastError();
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  SG_TRY_CUDA(le);
  const double fmas = (double)grid * 256 * CHAINS * 8 * (double)iters;
  *flops_per_s = ms > 0.f ? 2.0 * fmas / (ms * 1e-3) : 0.0;
  return SG_OK;
}

}  // namespace sghsc

extern "C" int sg_measure_alu_peak(int dtype, int iters, double* flops_per_s, void* stream) {
  sghsc::set_error("");
  if (!flops_per_s || iters < 1 || (dtype != SG_F64 && dtype != SG_F32)) {
    sghsc::set_error("sg_measure_alu_peak: invalid arguments");
    return SG_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == SG_F64) return sghsc::run_probe<double>(iters, flops_per_s, s);
  return sghsc::run_probe<float>(iters, flops_per_s, s);
}
