// Measured float32 CUDA-core peak.  The blur and channel-gradient kernels sit
// near the float32 ridge of GB300, so their rooflines need the FMA rate of
// the part as it runs, not a nominal figure: a kernel of independent FMA
// chains (eight per thread, no memory traffic) timed with CUDA events.
#include <algorithm>

#include "adjwt_internal.h"

namespace adjwt {
namespace {

__device__ float g_fma_sink;

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1e-3f * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s != s) g_fma_sink = s;  // never true for these inputs; keeps the chains live
}

}  // namespace
}  // namespace adjwt

using namespace adjwt;

extern "C" int adjwt_fp32_fma_peak(double* tflops, adjwt_stream_t stream) {
  if (!tflops) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_fp32_fma_peak: tflops is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int per_sm = 0;
  ADJWT_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe, kProbeThreads, 0));
  const int blocks = std::max(1, per_sm) * sm_count();
  const int iters = 4096;
  cudaEvent_t e0, e1;
  ADJWT_CUDA_CHECK(cudaEventCreate(&e0));
  ADJWT_CUDA_CHECK(cudaEventCreate(&e1));
  float best = 1e30f;
  int rc = ADJWT_OK;
  for (int rep = 0; rep < 6 && rc == ADJWT_OK; ++rep) {
    cudaError_t e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
      k_fma_probe<<<blocks, kProbeThreads, 0, s>>>(iters, 0.999999f, 1e-7f);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "adjwt_fp32_fma_peak");
    } else if (rep > 0) {  // the first launch warms up
      best = std::min(best, ms);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  const double flops = 2.0 * kChains * kUnroll * (double)iters * blocks * kProbeThreads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return ADJWT_OK;
}
