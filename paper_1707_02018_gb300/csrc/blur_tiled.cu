// Fused R^*(R u - b) without scratch as one tiled kernel (one 64 x 64 output
// tile per CTA; the tile body and its geometry are in blur_tile.cuh), for
// PSF radii up to kTiledMaxRadius.  Used when the persistent TMA passes
// (blur_tma.cu) cannot run or no scratch image is given.
#include <algorithm>

#include "adjwt_internal.h"
#include "blur_tile.cuh"
#include "device_common.cuh"

namespace adjwt {

namespace {

template <int R>
__global__ void __launch_bounds__(kNT) k_blur_normal_t(const TiledArgs a) {
  pdl_entry();
  extern __shared__ float sm[];
  __shared__ double red[kNT / 32];
  __shared__ int s_border;
  float sq = 0.0f;  // per-thread float32 partial, float64 across the block
  blur_normal_tile<R>(a, blockIdx.y, blockIdx.x, sm, &s_border, sq);
  if (a.partials) {
    const double tot = block_sum<kNT>((double)sq, red);
    if (threadIdx.x == 0) a.partials[blockIdx.y * gridDim.x + blockIdx.x] = 0.5 * tot;
  }
}

template <int R>
size_t smem_normal_t() {
  return blur_tile_smem<R>();
}
template <int R>
int launch_r(const TiledArgs& a, cudaStream_t s) {
  dim3 grid((a.cols + kT - 1) / kT, (a.rows + kT - 1) / kT);
  const size_t sm = smem_normal_t<R>();
  ADJWT_CUDA_CHECK(set_smem(k_blur_normal_t<R>, sm));
  ADJWT_TRACED("blur_normal", 0, s, pdl_launch(k_blur_normal_t<R>, grid, kNT, sm, s, a));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  return ADJWT_OK;
}

}  // namespace

int tiled_blur_grid_slots(const adjwt_blur_plan* p) {
  return ((p->cols + kT - 1) / kT) * ((p->rows + kT - 1) / kT);
}

bool tiled_blur_supported(const adjwt_blur_plan* p) {
  return (p->kr / 2) <= kTiledMaxRadius && (p->kc / 2) <= kTiledMaxRadius;
}

// Fused g = R^*(R u - b) in one kernel (no scratch image).
int launch_tiled_blur(const adjwt_blur_plan* p, const float* in, const float* b, float* out, double* partials,
                      cudaStream_t s) {
  const int R = std::max(p->kr / 2, p->kc / 2);
  TiledArgs a{};
  a.in = in;
  a.b = b;
  a.out = out;
  a.partials = partials;
  a.status = device_status_ptr();
  a.rows = p->rows;
  a.cols = p->cols;
  a.pitch = p->image_pitch;
  a.bc = p->bc;
  const int or_ = R - p->kr / 2, oc = R - p->kc / 2;
  for (int t = 0; t < p->kr; ++t) a.pr[or_ + t] = static_cast<float>(p->taps_r[t]);
  for (int t = 0; t < p->kc; ++t) a.pc[oc + t] = static_cast<float>(p->taps_c[t]);
  switch (R) {
#define ADJWT_R(r) \
  case r:          \
    return launch_r<r>(a, s);
    ADJWT_R(0) ADJWT_R(1) ADJWT_R(2) ADJWT_R(3) ADJWT_R(4) ADJWT_R(5) ADJWT_R(6)
    ADJWT_R(7) ADJWT_R(8) ADJWT_R(9) ADJWT_R(10) ADJWT_R(11) ADJWT_R(12)
#undef ADJWT_R
    default:
      return fail(ADJWT_ERR_INVALID_ARG, "tiled blur: radius above 12");
  }
}

}  // namespace adjwt
