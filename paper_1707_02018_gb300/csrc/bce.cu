// Gradient of the smooth part of the augmented multichannel blind channel
// problem (Sec. II, Eq. 6): C channels h_c (length k) share one source s
// (length n), observations x_c (length n + k - 1), r_c = h_c * s - x_c:
//   f = sum_c ||r_c||^2 + (lambda_tv / delta) L_delta(D h_c),
//   grad_{h_c} = 2 S^T r_c + (lambda_tv / delta) D^T clip(D h_c, -delta, delta),
//   grad_s     = sum_c 2 H_c^T r_c,
// with (D h)[j] = h[j+1] - h[j] and L_delta the Huber function.  The
// correlations come from the channel-gradient kernels (one row per channel,
// the source replicated into the workspace); one more kernel scales them,
// adds the softened-TV term and sums the source gradient over the channels.
#include "adjwt_internal.h"

namespace adjwt {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float clip(float z, float d) { return fminf(fmaxf(z, -d), d); }

__global__ void __launch_bounds__(kThreads) k_bce_finish(int C, int64_t n, int k, const float* __restrict__ h,
                                                         float* __restrict__ grad_h,
                                                         const float* __restrict__ gs_rows,
                                                         float* __restrict__ grad_s, float w_tv, float delta) {
  pdl_entry();
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (grad_s && i < n) {
    float acc = 0.0f;
    for (int c = 0; c < C; ++c) acc += gs_rows[(size_t)c * n + i];
    grad_s[i] = 2.0f * acc;
  }
  if (grad_h && i < (int64_t)C * k) {
    const int c = static_cast<int>(i / k), j = static_cast<int>(i - (int64_t)c * k);
    const float* hc = h + (size_t)c * k;
    const float prev = j > 0 ? clip(hc[j] - hc[j - 1], delta) : 0.0f;      // (D h)[j-1]
    const float cur = j < k - 1 ? clip(hc[j + 1] - hc[j], delta) : 0.0f;   // (D h)[j]
    grad_h[i] = 2.0f * grad_h[i] + w_tv * (prev - cur);
  }
}

}  // namespace

int launch_bce_finish(int C, int64_t n, int k, const float* h, float* grad_h, const float* gs_rows, float* grad_s,
                      double lambda_tv, double delta, cudaStream_t s) {
  const int64_t count = std::max<int64_t>(n, (int64_t)C * k);
  const unsigned nb = static_cast<unsigned>((count + kThreads - 1) / kThreads);
  ADJWT_TRACED("bce_finish", 0, s,
               pdl_launch(k_bce_finish, nb, kThreads, 0, s, C, n, k, h, grad_h, gs_rows, grad_s,
                          static_cast<float>(lambda_tv / delta), static_cast<float>(delta)));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  return ADJWT_OK;
}

}  // namespace adjwt
