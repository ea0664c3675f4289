// FP32 FMA rate of the device: the denominator of the ALU roofline that the
// FP32 correlation kernel is measured against.  Every thread runs 8 independent
// FMA chains (enough to cover the FMA latency at 4 warps per scheduler), so the
// rate is the FMA pipes' throughput, not their latency.
#include "vimg_internal.h"

namespace vimg {

constexpr int kPeakThreads = 512, kPeakChains = 8;

__global__ void __launch_bounds__(kPeakThreads) k_fma_rate(int iters, float seed, float* sink) {
  float a[kPeakChains];
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) a[c] = seed + 0.001f * (threadIdx.x + c);
  const float m = 0.9999999f, k = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int c = 0; c < kPeakChains; ++c) a[c] = fmaf(a[c], m, k);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kPeakChains; ++c) s += a[c];
  if (s == 12345.678f) sink[blockIdx.x] = s;  // never true; keeps the chains live
}

}  // namespace vimg

extern "C" int vimg_fma_rate(void* stream, double* flops_per_s) {
  using namespace vimg;
  if (!flops_per_s) return VIMG_ERR_ARG;
  const int sms = sm_count();
  if (sms <= 0) return VIMG_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int blocks = 2 * sms, iters = 4096;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return VIMG_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return VIMG_ERR_CUDA;
  }
  int rc = VIMG_OK;
  float ms = 0.f;
  for (int rep = 0; rep < 3 && rc == VIMG_OK; ++rep) {  // the first run warms up
    if (cudaEventRecord(e0, st) != cudaSuccess) rc = VIMG_ERR_CUDA;
    k_fma_rate<<<blocks, kPeakThreads, 0, st>>>(iters, 1.0f, nullptr);
    if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
        cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      rc = VIMG_ERR_CUDA;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != VIMG_OK || ms <= 0.f) return rc == VIMG_OK ? VIMG_ERR_CUDA : rc;
  const double fmas = (double)blocks * kPeakThreads * iters * 16.0 * kPeakChains;
  *flops_per_s = 2.0 * fmas / (ms * 1e-3);
  return VIMG_OK;
}
