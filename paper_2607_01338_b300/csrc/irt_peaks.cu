// Microbenchmark of the two pipes that bound the transfer kernels (FP32 FMA
// and the special-function unit), measured on the running device at its
// present clock; the roofline denominators of the measurement harness.
#include <cuda_runtime.h>

#include <algorithm>

#include "irt_internal.h"

namespace irt {
namespace dev {

constexpr int kChains = 8;    // independent dependency chains per thread
constexpr int kPeakIters = 2048;

__global__ void __launch_bounds__(256) fma_peak_kernel(float* sink, float m, float c) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (float)(threadIdx.x + i) * 1e-3f;
#pragma unroll 16
  for (int it = 0; it < kPeakIters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], m, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) ex2_peak_kernel(float* sink) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (float)(threadIdx.x + i) * 1e-3f;
#pragma unroll 16
  for (int it = 0; it < kPeakIters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      // 2^-a stays in (0, 1] for a in [0, 1]
      asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(a[i]) : "f"(-a[i]));
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace dev
}  // namespace irt

extern "C" irt_status irt_measure_pipe_peaks(double* fp32_ops_per_s, double* mufu_ops_per_s,
                                             void* cuda_stream) {
  if (!fp32_ops_per_s || !mufu_ops_per_s) return IRT_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256, blocks = std::max(sms, 1) * 8;
  float* sink = nullptr;
  if (cudaMalloc((void**)&sink, sizeof(float) * (size_t)threads * blocks) != cudaSuccess) {
    cudaGetLastError();
    return IRT_ENOMEM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const double ops = (double)threads * blocks * irt::dev::kPeakIters * irt::dev::kChains;
  double best_fma = 0.0, best_ex2 = 0.0;
  irt_status st = IRT_OK;
  for (int rep = 0; rep < 4 && st == IRT_OK; ++rep) {
    for (int which = 0; which < 2; ++which) {
      cudaEventRecord(e0, s);
      if (which == 0)
        irt::dev::fma_peak_kernel<<<blocks, threads, 0, s>>>(sink, 0.9990234375f, 1e-3f);
      else
        irt::dev::ex2_peak_kernel<<<blocks, threads, 0, s>>>(sink);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        st = IRT_ECUDA;
        break;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      const double rate = ops / ((double)ms * 1e-3);
      if (rep > 0) {   // the first round warms up
        if (which == 0) best_fma = std::max(best_fma, rate);
        else best_ex2 = std::max(best_ex2, rate);
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  *fp32_ops_per_s = best_fma;
  *mufu_ops_per_s = best_ex2;
  return st;
}
