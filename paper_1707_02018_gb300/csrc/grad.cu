// Kernels for differentiating through the FISTA iteration (unrolled FISTA,
// gradients with respect to lambda, the PSF width sigma and the data b).
//
// The backward of one iteration x_{k+1} = S_tau(y_k - (1/L) A^*(A y_k - b)),
// A = R W (Sec. 1, Eq. 1), needs, besides the operators W, W^*, R and R^*
// themselves (their exactness is what makes the chain rule A^* grad l(A x)
// correct, Sec. 1), only elementwise pieces:
//   * the soft-threshold's vector-Jacobian product: zbar = xbar [x_{k+1} != 0]
//     and d/dtau = -sum sign(x_{k+1}) xbar (S_tau(z) = 0 exactly when
//     |z| <= tau, and there its derivative is 0);
//   * a x + b y for the momentum and step terms;
//   * float64 inner products of images or coefficient vectors (for the
//     scalar gradients), with per-block float64 partials added in a fixed
//     order, so results are reproducible.
#include <algorithm>
#include <cmath>

#include "adjwt_internal.h"
#include "device_common.cuh"

namespace adjwt {
namespace {

constexpr int kThreads = 256;
constexpr int kDotBlocks = 608;  // 4 x 152 SMs: partial slots of one inner product

// out = a x + b y on rows x cols of arrays with row pitch `pitch` (pitch
// columns beyond cols untouched); a flat vector is rows = 1, cols = pitch = n
__global__ void __launch_bounds__(kThreads) k_axpby(int rows, int64_t cols, int64_t pitch, float a,
                                                    const float* __restrict__ x, float b,
                                                    const float* __restrict__ y, float* __restrict__ out) {
  pdl_entry();
  const int64_t n = (int64_t)rows * cols;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    const int64_t r = i / cols, o = r * pitch + (i - r * cols);
    out[o] = fmaf(a, x[o], b * y[o]);
  }
}

// out = S_tau(in): the soft threshold of the FISTA prox (|v| <= tau -> 0)
__global__ void __launch_bounds__(kThreads) k_soft(int64_t n, const float* __restrict__ in, float tau,
                                                   float* __restrict__ out) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    const float v = in[i], mag = fabsf(v) - tau;
    out[i] = mag > 0.0f ? copysignf(mag, v) : 0.0f;
  }
}

// partials[block] = sum over the block's elements of x y (rows x cols of a pitched array)
__global__ void __launch_bounds__(kThreads) k_dot(int rows, int64_t cols, int64_t pitch, const float* __restrict__ x,
                                                  const float* __restrict__ y, double* __restrict__ partials) {
  pdl_entry();
  __shared__ double red[kThreads / 32];
  const int64_t total = (int64_t)rows * cols;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < total; i += (int64_t)gridDim.x * kThreads) {
    const int64_t r = i / cols, c = i - r * cols;
    acc += (double)x[r * pitch + c] * (double)y[r * pitch + c];
  }
  const double t = block_sum<kThreads>(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// zbar = xbar [x_next != 0]; partials[block] = sum sign(x_next) xbar
__global__ void __launch_bounds__(kThreads) k_prox_vjp(int64_t n, const float* __restrict__ x_next,
                                                       const float* __restrict__ xbar, float* __restrict__ zbar,
                                                       double* __restrict__ partials) {
  pdl_entry();
  __shared__ double red[kThreads / 32];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    const float x = x_next[i], g = xbar[i];
    const bool on = x != 0.0f;
    zbar[i] = on ? g : 0.0f;
    if (on) acc += x > 0.0f ? (double)g : -(double)g;
  }
  const double t = block_sum<kThreads>(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

unsigned grid_for(int64_t n) {
  const int64_t b = (n + kThreads - 1) / kThreads;
  return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(b, kDotBlocks)));
}

}  // namespace

int launch_axpby(int rows, int64_t cols, int64_t pitch, float a, const float* x, float b, const float* y, float* out,
                 cudaStream_t st) {
  ADJWT_TRACED("axpby", 0, st,
               pdl_launch(k_axpby, grid_for((int64_t)rows * cols), kThreads, 0, st, rows, cols, pitch, a, x, b, y, out));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  return ADJWT_OK;
}

int launch_dot_partials(int rows, int64_t cols, int64_t pitch, const float* x, const float* y, double* partials,
                        cudaStream_t st, int* nparts) {
  const unsigned nb = grid_for((int64_t)rows * cols);
  ADJWT_TRACED("dot", 0, st, pdl_launch(k_dot, nb, kThreads, 0, st, rows, cols, pitch, x, y, partials));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  *nparts = static_cast<int>(nb);
  return ADJWT_OK;
}

int launch_prox_vjp_partials(int64_t n, const float* x_next, const float* xbar, float* zbar, double* partials,
                             cudaStream_t st, int* nparts) {
  const unsigned nb = grid_for(n);
  ADJWT_TRACED("prox_vjp", 0, st, pdl_launch(k_prox_vjp, nb, kThreads, 0, st, n, x_next, xbar, zbar, partials));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  *nparts = static_cast<int>(nb);
  return ADJWT_OK;
}

size_t reduce_partials_bytes() { return (size_t)kDotBlocks * sizeof(double); }

}  // namespace adjwt

using namespace adjwt;

extern "C" size_t adjwt_reduce_workspace_size(void) { return reduce_partials_bytes(); }

extern "C" int adjwt_axpby(int64_t n, float a, const float* x, float b, const float* y, float* out,
                           adjwt_stream_t stream) {
  if (n < 0) return fail(ADJWT_ERR_SHAPE, "adjwt_axpby: n < 0");
  if (n == 0) return ADJWT_OK;
  if (!x || !y || !out) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_axpby: NULL pointer");
  return launch_axpby(1, n, n, a, x, b, y, out, stream);
}

extern "C" int adjwt_soft_threshold(int64_t n, const float* in, double tau, float* out, adjwt_stream_t stream) {
  if (n < 0) return fail(ADJWT_ERR_SHAPE, "adjwt_soft_threshold: n < 0");
  if (n == 0) return ADJWT_OK;
  if (!in || !out) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_soft_threshold: NULL pointer");
  if (!(tau >= 0.0) || !std::isfinite(tau)) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_soft_threshold: need finite tau >= 0");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned nb = static_cast<unsigned>(std::min<int64_t>((n + kThreads - 1) / kThreads, 4 * 152));
  ADJWT_TRACED("soft_threshold", 0, st, pdl_launch(k_soft, nb, kThreads, 0, st, n, in, static_cast<float>(tau), out));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  return ADJWT_OK;
}

extern "C" int adjwt_dot(int rows, int64_t cols, int64_t pitch, const float* x, const float* y, double* out_dev,
                         void* ws, size_t ws_bytes, adjwt_stream_t stream) {
  if (rows < 0 || cols < 0 || pitch < cols) return fail(ADJWT_ERR_SHAPE, "adjwt_dot: need rows, cols >= 0, pitch >= cols");
  if (!x || !y || !out_dev) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_dot: NULL pointer");
  if (!ws || ws_bytes < adjwt_reduce_workspace_size())
    return fail(ADJWT_ERR_WORKSPACE, "adjwt_dot: workspace of adjwt_reduce_workspace_size() bytes needed");
  auto* part = static_cast<double*>(ws);
  int nb = 0;
  int rc = launch_dot_partials(rows, cols, pitch, x, y, part, stream, &nb);
  if (rc) return rc;
  return launch_sum_partials(part, nb, 1.0, nullptr, 0, 0.0, out_dev, stream);
}

extern "C" int fista_prox_vjp(int64_t n, const float* x_next, const float* xbar, float* zbar, double* sign_dot_dev,
                              void* ws, size_t ws_bytes, adjwt_stream_t stream) {
  if (n < 0) return fail(ADJWT_ERR_SHAPE, "fista_prox_vjp: n < 0");
  if (!x_next || !xbar || !zbar || !sign_dot_dev) return fail(ADJWT_ERR_INVALID_ARG, "fista_prox_vjp: NULL pointer");
  if (!ws || ws_bytes < adjwt_reduce_workspace_size())
    return fail(ADJWT_ERR_WORKSPACE, "fista_prox_vjp: workspace of adjwt_reduce_workspace_size() bytes needed");
  auto* part = static_cast<double*>(ws);
  int nb = 0;
  int rc = launch_prox_vjp_partials(n, x_next, xbar, zbar, part, stream, &nb);
  if (rc) return rc;
  return launch_sum_partials(part, nb, 1.0, nullptr, 0, 0.0, sign_dot_dev, stream);
}
