// Device status word and TMA descriptor encoding.
//
// Kernels that wait on asynchronous copies record ADJWT_ERR_TIMEOUT here when
// a bounded wait gives up; adjwt_device_status() reads (and optionally
// clears) it.  Tensor maps are encoded through the runtime's driver entry
// point, so the library does not link against libcuda directly.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <vector>

#include "adjwt_internal.h"
#include "tma.cuh"

namespace adjwt {
namespace {

__device__ int g_device_status;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int* g_status_ptr[kMaxDevices] = {};

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

}  // namespace

namespace {
struct SmemAttr {
  const void* kernel;
  int device;
  size_t bytes;
};
std::mutex g_attr_mu;
std::vector<SmemAttr> g_attrs;
}  // namespace

bool smem_attr_known(const void* kernel, size_t bytes, bool mark) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  std::lock_guard<std::mutex> lock(g_attr_mu);
  for (auto& a : g_attrs)
    if (a.kernel == kernel && a.device == dev) {
      if (a.bytes >= bytes) return true;
      if (mark) {
        a.bytes = bytes;
        return true;
      }
      return false;
    }
  if (mark) g_attrs.push_back({kernel, dev, bytes});
  return mark;
}

int* device_status_ptr() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_status_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_status) != cudaSuccess) return nullptr;
    g_status_ptr[dev] = static_cast<int*>(p);
  }
  return g_status_ptr[dev];
}

int make_tmap_2d_f32(CUtensorMap* map, const float* base, int rows, int cols, int pitch_floats, int box_rows,
                     int box_cols) {
  return make_tmap_2d_f32_sw(map, base, rows, cols, pitch_floats, box_rows, box_cols, false);
}

int make_tmap_2d_f32_sw(CUtensorMap* map, const float* base, int rows, int cols, int pitch_floats, int box_rows,
                        int box_cols, bool swizzle128) {
  auto fn = encode_fn();
  if (!fn) return fail(ADJWT_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(pitch_floats) * sizeof(float)};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(box_cols), static_cast<cuuint32_t>(box_rows)};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ADJWT_ERR_CUDA, "cuTensorMapEncodeTiled failed (code " + std::to_string(r) + ")");
  return ADJWT_OK;
}

int sm_count() {
  static int n[kMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 1;
  if (!n[dev]) {
    int v = 1;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    n[dev] = v > 0 ? v : 1;
  }
  return n[dev];
}

}  // namespace adjwt

using namespace adjwt;

extern "C" int adjwt_device_status(int* status_out, int clear) {
  if (!status_out) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_device_status: status_out is NULL");
  int v = 0;
  ADJWT_CUDA_CHECK(cudaMemcpyFromSymbol(&v, g_device_status, sizeof(int)));
  if (clear) {
    const int zero = 0;
    ADJWT_CUDA_CHECK(cudaMemcpyToSymbol(g_device_status, &zero, sizeof(int)));
  }
  *status_out = v;
  return ADJWT_OK;
}

// Self-test of the bounded wait that every asynchronous-copy and tensor-core
// completion wait of the library uses (mbar_wait: about one second of SM
// cycles).  One thread arms a barrier that expects one arrival; with
// arrive != 0 it arrives itself and the wait returns at once, otherwise
// nothing ever completes the barrier, the wait gives up at its limit and the
// kernel records ADJWT_ERR_TIMEOUT and returns normally.
namespace adjwt {
namespace {
__global__ void k_wait_selftest(int arrive, int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_mbar_init();
  if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
  if (!mbar_wait(&bar, 0)) record_status(status, ADJWT_ERR_TIMEOUT);
}
}  // namespace
}  // namespace adjwt

extern "C" int adjwt_wait_selftest(int arrive, adjwt_stream_t stream) {
  int* st = device_status_ptr();
  if (!st) return fail(ADJWT_ERR_CUDA, "adjwt_wait_selftest: no device status word");
  k_wait_selftest<<<1, 32, 0, stream>>>(arrive, st);
  ADJWT_CUDA_CHECK(cudaGetLastError());
  return ADJWT_OK;
}
