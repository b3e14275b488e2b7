// Blind-channel gradients of Sec. II (Eq. 5), batched over independent rows.
//
//   grad_s[m] = sum_{i<K} h[i] r[i+m]   (m < N)   -- H^T r, valid correlation
//   grad_h[j] = sum_{i<N} s[i] r[i+j]   (j < K)   -- S^T r, valid correlation
//   r = h * s - x                                  -- the residual (full conv)
//
// One CTA owns a chunk of kChunk samples of one row: it stages r (with the
// K-1 tail), s and h in shared memory, writes grad_s for its chunk and a
// partial grad_h over its chunk to workspace; a second pass sums the partials
// of each row in a fixed order (deterministic, no atomics).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "adjwt_internal.h"
#include "device_common.cuh"

namespace adjwt {
namespace {

constexpr int kChunk = 1024;
constexpr int kThreads = 256;
constexpr int kMaxK = 4096;

__global__ void __launch_bounds__(kThreads) k_conv_adjoint(int64_t n, int K, const float* __restrict__ s,
                                                           const float* __restrict__ h, const float* __restrict__ r,
                                                           float* __restrict__ grad_s, float* __restrict__ part_h,
                                                           int nchunks) {
  pdl_entry();
  extern __shared__ float sm[];
  float* rs = sm;                    // kChunk + K - 1
  float* ss = rs + kChunk + K - 1;   // kChunk
  float* hs = ss + kChunk;           // K
  float* red = hs + K;               // kThreads
  const int b = blockIdx.y;
  const int64_t m0 = (int64_t)blockIdx.x * kChunk;
  const int64_t nr = n + K - 1;
  const float* rrow = r + (size_t)b * nr;
  const float* srow = s + (size_t)b * n;
  const int tid = threadIdx.x;
  for (int i = tid; i < kChunk + K - 1; i += kThreads) {
    const int64_t g = m0 + i;
    rs[i] = g < nr ? __ldg(rrow + g) : 0.0f;
  }
  for (int i = tid; i < kChunk; i += kThreads) {
    const int64_t g = m0 + i;
    ss[i] = g < n ? __ldg(srow + g) : 0.0f;
  }
  if (h)
    for (int i = tid; i < K; i += kThreads) hs[i] = __ldg(h + (size_t)b * K + i);
  __syncthreads();

  if (grad_s) {
    float acc[kChunk / kThreads];
#pragma unroll
    for (int q = 0; q < kChunk / kThreads; ++q) acc[q] = 0.0f;
    for (int i = 0; i < K; ++i) {
      const float hv = hs[i];
#pragma unroll
      for (int q = 0; q < kChunk / kThreads; ++q) acc[q] = fmaf(hv, rs[tid + q * kThreads + i], acc[q]);
    }
    float* out = grad_s + (size_t)b * n;
#pragma unroll
    for (int q = 0; q < kChunk / kThreads; ++q) {
      const int64_t m = m0 + tid + q * kThreads;
      if (m < n) out[m] = acc[q];
    }
  }

  if (part_h) {
    // lags are spread over the threads; each lag's sample range is split in P parts
    const int P = K >= kThreads ? 1 : kThreads / K;
    const int span = (kChunk + P - 1) / P;
    float* dst = part_h + ((size_t)b * nchunks + blockIdx.x) * K;
    for (int j0 = 0; j0 < K; j0 += kThreads / P) {
      const int j = j0 + tid % (kThreads / P);
      const int part = tid / (kThreads / P);
      float acc = 0.0f;
      if (j < K && part < P) {
        const int i0 = part * span, i1 = min(kChunk, i0 + span);
        for (int i = i0; i < i1; ++i) acc = fmaf(ss[i], rs[i + j], acc);
      }
      red[tid] = acc;
      __syncthreads();
      if (tid < kThreads / P && j0 + tid < K) {
        float t = 0.0f;
        for (int p = 0; p < P; ++p) t += red[p * (kThreads / P) + tid];
        dst[j0 + tid] = t;
      }
      __syncthreads();
    }
  }
}

__global__ void k_conv_reduce(int K, int nchunks, const float* __restrict__ part_h, float* __restrict__ grad_h,
                              int64_t total) {
  pdl_entry();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int64_t b = idx / K;
  const int j = static_cast<int>(idx - b * K);
  const float* p = part_h + (size_t)b * nchunks * K + j;
  float acc = 0.0f;
  for (int c = 0; c < nchunks; ++c) acc += p[(size_t)c * K];
  grad_h[idx] = acc;
}

__global__ void __launch_bounds__(kThreads) k_conv_residual(int64_t n, int K, const float* __restrict__ h,
                                                            const float* __restrict__ s, const float* __restrict__ x,
                                                            float* __restrict__ r) {
  pdl_entry();
  extern __shared__ float sm[];
  float* seg = sm;                  // s[m0 - K + 1 .. m0 + kChunk)
  float* hs = seg + kChunk + K - 1;
  const int b = blockIdx.y;
  const int64_t m0 = (int64_t)blockIdx.x * kChunk;
  const int64_t nr = n + K - 1;
  const int tid = threadIdx.x;
  for (int i = tid; i < kChunk + K - 1; i += kThreads) {
    const int64_t g = m0 - (K - 1) + i;
    seg[i] = (g >= 0 && g < n) ? __ldg(s + (size_t)b * n + g) : 0.0f;
  }
  for (int i = tid; i < K; i += kThreads) hs[i] = __ldg(h + (size_t)b * K + i);
  __syncthreads();
  for (int q = 0; q < kChunk / kThreads; ++q) {
    const int mm = tid + q * kThreads;
    const int64_t m = m0 + mm;
    if (m >= nr) break;
    float acc = 0.0f;
    for (int i = 0; i < K; ++i) acc = fmaf(hs[i], seg[mm + K - 1 - i], acc);
    if (x) acc -= __ldg(x + (size_t)b * nr + m);
    r[(size_t)b * nr + m] = acc;
  }
}

int64_t nchunks_of(int64_t n) { return (n + kChunk - 1) / kChunk; }

}  // namespace

void conv_reduce(unsigned nblocks, int k, int nchunks, const float* partials, float* grad_h, int64_t total,
                 cudaStream_t st) {
  pdl_launch(k_conv_reduce, nblocks, 256, 0, st, k, nchunks, partials, grad_h, total);
}

int64_t conv_partial_floats(int batch, int64_t n, int k) {
  if (conv_fused_supported(k)) return (int64_t)batch * conv_fused_nchunks(n, k) * k;
  return (int64_t)batch * nchunks_of(n) * k;
}

int launch_conv_adjoint(int batch, int64_t n, int k, const float* s, const float* h, const float* r, float* grad_h,
                        float* grad_s, float* partials, cudaStream_t st) {
  if (k > kMaxK) return fail(ADJWT_ERR_SHAPE, "conv_adjoint: k above 4096");
  if (batch == 0) return ADJWT_OK;
  if (conv_fused_supported(k))
    return launch_conv_fused(batch, n, k, s, h, nullptr, r, nullptr, grad_h, grad_s, partials, st);
  const int64_t nch = nchunks_of(n);
  if (nch > 65535 * 1024LL) return fail(ADJWT_ERR_SHAPE, "conv_adjoint: n too large");
  const size_t smem = (size_t)(kChunk + k - 1 + kChunk + k + kThreads) * sizeof(float);
  if (smem > 48 * 1024)
    ADJWT_CUDA_CHECK(cudaFuncSetAttribute(k_conv_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          static_cast<int>(smem)));
  dim3 grid(static_cast<unsigned>(nch), static_cast<unsigned>(batch));
  ADJWT_TRACED("conv_adjoint", 0, st,
               pdl_launch(k_conv_adjoint, grid, kThreads, smem, st, n, k, s, h, r, grad_s, grad_h ? partials : nullptr,
                                                            static_cast<int>(nch)));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  if (grad_h) {
    const int64_t total = (int64_t)batch * k;
    const unsigned nb = static_cast<unsigned>((total + 255) / 256);
    ADJWT_TRACED("conv_reduce", 0, st,
                 pdl_launch(k_conv_reduce, nb, 256, 0, st, k, static_cast<int>(nch), partials, grad_h, total));
    ADJWT_CUDA_CHECK(cudaGetLastError());
  }
  return ADJWT_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of conv_adjoint.  Some callers must not allocate
// device memory on their call path: processes whose device memory belongs to
// another allocator (a framework's pool or a fixed budget), loops where the
// device-wide synchronisation of cudaMalloc / cudaFree is not acceptable, and
// deployments that forbid allocation after start-up.  For them the grad_h
// partial sums live in a fixed array in this library's device memory instead
// of a caller workspace.  The array is loaded with the library's module, so
// every GPU that loads the library holds it until the process exits.
namespace {

constexpr int64_t kStaticScratchFloats = int64_t(1) << 20;  // 4 MiB
__device__ __align__(256) float g_conv_static_scratch[kStaticScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
struct StaticSlot {
  unsigned long long ctx_id;  // unique for the life of the process (cuCtxGetId)
  float* ptr;
};
StaticSlot g_static_slot[kMaxDevices] = {};


template <class F>
F driver_fn(const char* name, int version) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  if (cudaGetDriverEntryPointByVersion(name, &p, version, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return nullptr;
  return reinterpret_cast<F>(p);
}

// Identifier of the context current on this thread (0 if none is current yet).
int current_ctx_id(unsigned long long* id) {
  static const auto get_ctx = driver_fn<PFN_cuCtxGetCurrent_v4000>("cuCtxGetCurrent", 4000);
  static const auto get_id = driver_fn<PFN_cuCtxGetId_v12000>("cuCtxGetId", 12000);
  if (!get_ctx || !get_id) return fail(ADJWT_ERR_CUDA, "conv_adjoint_noalloc: cuCtxGetCurrent/cuCtxGetId unavailable");
  CUcontext ctx = nullptr;
  if (get_ctx(&ctx) != CUDA_SUCCESS) return fail(ADJWT_ERR_CUDA, "conv_adjoint_noalloc: cuCtxGetCurrent failed");
  *id = 0;
  if (ctx && get_id(ctx, id) != CUDA_SUCCESS) return fail(ADJWT_ERR_CUDA, "conv_adjoint_noalloc: cuCtxGetId failed");
  return ADJWT_OK;
}

// Device address of the array in the current context.  In host code the
// array's name is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress, with the device current, the first time a context uses
// the entry point, and cached under that context's process-unique id: a new
// context (after cudaDeviceReset, or a non-primary context made current) loads
// the module again, possibly elsewhere, and gets its own lookup.
int static_scratch(float** out) {
  int dev = 0;
  ADJWT_CUDA_CHECK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(ADJWT_ERR_INVALID_ARG, "conv_adjoint_noalloc: device index above 63");
  unsigned long long id = 0;
  int rc = current_ctx_id(&id);
  if (rc) return rc;
  std::lock_guard<std::mutex> lock(g_static_mu);
  StaticSlot& slot = g_static_slot[dev];
  if (id == 0 || slot.ctx_id != id || !slot.ptr) {
    void* p = nullptr;
    ADJWT_CUDA_CHECK(cudaGetSymbolAddress(&p, g_conv_static_scratch));  // makes the primary context current if none was
    rc = current_ctx_id(&id);
    if (rc) return rc;
    slot.ctx_id = id;
    slot.ptr = static_cast<float*>(p);
  }
  *out = slot.ptr;
  return ADJWT_OK;
}

}  // namespace

int64_t conv_static_scratch_floats() { return kStaticScratchFloats; }

int launch_conv_adjoint_noalloc(int batch, int64_t n, int k, const float* s, const float* h, const float* r,
                                float* grad_h, float* grad_s, cudaStream_t st) {
  float* scratch = nullptr;
  if (grad_h) {
    int rc = static_scratch(&scratch);
    if (rc) return rc;
  }
  // Every (row, chunk, lag) slot the reduction reads is written by exactly one
  // CTA of the same call, so nothing has to be cleared between calls.
  return launch_conv_adjoint(batch, n, k, s, h, r, grad_h, grad_s, scratch, st);
}

int launch_conv_residual(int batch, int64_t n, int k, const float* h, const float* s, const float* x, float* r,
                         cudaStream_t st) {
  if (k > kMaxK) return fail(ADJWT_ERR_SHAPE, "conv_residual: k above 4096");
  if (batch == 0) return ADJWT_OK;
  const int64_t nr = n + k - 1;
  const size_t smem = (size_t)(kChunk + k - 1 + k) * sizeof(float);
  if (smem > 48 * 1024)
    ADJWT_CUDA_CHECK(cudaFuncSetAttribute(k_conv_residual, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          static_cast<int>(smem)));
  dim3 grid(static_cast<unsigned>(nchunks_of(nr)), static_cast<unsigned>(batch));
  ADJWT_TRACED("conv_residual", 0, st, pdl_launch(k_conv_residual, grid, kThreads, smem, st, n, k, h, s, x, r));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  return ADJWT_OK;
}

}  // namespace adjwt
