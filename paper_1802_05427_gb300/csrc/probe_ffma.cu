// Measured FP32 FMA peak of the device (rapro_measure_ffma_peak).
//
// The FP32 part of the receive path (Gram, matched filter, factorisations, the FMA
// estimator kernels) is bounded by the rate of FP32 fused multiply-adds.  This probe
// measures that rate instead of deriving it from lane counts and the nominal clock: every
// thread of a full-occupancy grid runs kChains independent FMA recurrences
// a <- a * m + c (m, c kernel parameters, so nothing folds at compile time), enough
// independent work per scheduler to hide the FMA latency.  It uses none of the receive
// kernels and allocates nothing (the result sink is a file-scope device word).
#include <cuda_runtime.h>

#include "rapro_internal.h"

namespace rapro {
namespace {

constexpr int kChains = 8;          // independent recurrences per thread
constexpr int kUnroll = 16;         // FMA rounds per loop trip
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;     // 2048 threads per SM: full occupancy

static __device__ float g_ffma_sink;

__global__ void __launch_bounds__(kThreads) ffma_chain_kernel(float m, float c, int trips) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = float(threadIdx.x) * 1.0e-3f + float(k);
  for (int it = 0; it < trips; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.0f) g_ffma_sink = s;    // the sum is positive: never stored, but kept live
}

}  // namespace
}  // namespace rapro

using namespace rapro;

extern "C" rapro_status rapro_measure_ffma_peak(int trips, double* tflops_out, double* ms_out,
                                                rapro_stream stream) {
  if (trips < 1 || !tflops_out) {
    set_error("rapro_measure_ffma_peak: trips must be >= 1 and tflops_out non-NULL");
    return RAPRO_ERR_INVALID_ARG;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "device query");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const dim3 grid(sms * kBlocksPerSm), block(kThreads);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_fail(e, "cudaEventCreate");
  }
  // 0.999 and 1e-3 keep every recurrence near its fixed point 1: finite, no denormals.
  ffma_chain_kernel<<<grid, block, 0, st>>>(0.999f, 1.0e-3f, trips < 64 ? trips : 64);   // warm-up
  cudaEventRecord(e0, st);
  ffma_chain_kernel<<<grid, block, 0, st>>>(0.999f, 1.0e-3f, trips);
  cudaEventRecord(e1, st);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "FFMA probe");
  const double flops = 2.0 * double(kChains) * kUnroll * double(trips) * double(grid.x) * kThreads;
  *tflops_out = flops / (double(ms) * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
  return RAPRO_OK;
}
