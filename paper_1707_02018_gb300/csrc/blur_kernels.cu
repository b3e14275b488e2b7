// Blur R, its adjoint R^*, and the fused data gradient R^*(R u - b).
//
// Per axis (PSF taps p[0..2r], Sec. I):
//     (R u)[i]   = sum_a p[a] u[ext(i + r - a)]
//     (R^* v)[j] = sum_{x : ext(x) = j} sum_a p[a] v0[x - r + a]     (v0 = 0 off-image)
// with ext the zero / half-point symmetric / circular extension.  The fold
// over copies is rewritten as a gather so that every output is owned by one
// thread:
//     (R^* v)[j] = sum_a p'[a] v[ext(j - r + a)],
//     p'[a] = p[2r - a] where the virtual sample j - r + a lies in an odd
//             (reflected) period of the symmetric extension, else p[a];
// for the zero extension v0 is used as is, for the circular one p' = p.
// (This is the transpose of the reflection written sample by sample.)
// Tiles of kTile x kTile outputs stage the boundary-extended input in shared
// memory (extension in the load path), then run the column and row passes.
// The fused kernel keeps R u - b in shared memory between R and R^*.
#include <algorithm>

#include "adjwt_internal.h"
#include "device_common.cuh"

namespace adjwt {
namespace {

constexpr int kTile = 32;
constexpr int kThreads = 256;
constexpr int kMaxK = 2 * kMaxBlurRadius + 1;

struct BlurArgs {
  const float* in;  // u (forward / normal) or v (adjoint)
  const float* b;   // observed image (normal / residual), may be null
  float* out;       // null for the residual-norm-only variant
  double* partials; // per-CTA 1/2 sum (Ru-b)^2, may be null
  int rows, cols, pitch, bc;
  int rr, rc;       // radii
  float pr[kMaxK], pc[kMaxK];
};

__device__ __forceinline__ bool odd_period(int x, int N) { return (floor_div(x, N) & 1) != 0; }

// Forward R (optionally minus b, optionally only the norm).
__global__ void __launch_bounds__(kThreads) k_blur_fwd(const BlurArgs a) {
  pdl_entry();
  extern __shared__ float sm[];
  const int rr = a.rr, rc = a.rc;
  const int UR = kTile + 2 * rr, UC = kTile + 2 * rc;
  float* U = sm;                 // UR x UC
  float* T1 = U + UR * UC;       // kTile x UC
  int* src_c = reinterpret_cast<int*>(T1 + kTile * UC);
  __shared__ double red[kThreads / 32];
  const int y0 = blockIdx.y * kTile, x0 = blockIdx.x * kTile;
  const int tid = threadIdx.x;
  for (int c = tid; c < UC; c += kThreads) src_c[c] = ext_src(x0 - rc + c, a.cols, a.bc == 3 ? 2 : a.bc);
  __syncthreads();
  for (int i = tid; i < UR * UC; i += kThreads) {
    const int u = i / UC, c = i - u * UC;
    const int sr = ext_src(y0 - rr + u, a.rows, a.bc == 3 ? 2 : a.bc), sc = src_c[c];
    U[i] = (sr >= 0 && sc >= 0) ? __ldg(a.in + (size_t)sr * a.pitch + sc) : 0.0f;
  }
  __syncthreads();
  for (int i = tid; i < kTile * UC; i += kThreads) {
    const int ii = i / UC, c = i - ii * UC;
    float acc = 0.0f;
    for (int t = 0; t <= 2 * rr; ++t) acc = fmaf(a.pr[t], U[(ii + 2 * rr - t) * UC + c], acc);
    T1[i] = acc;
  }
  __syncthreads();
  float sq = 0.0f;  // per-thread float32 partial, float64 across the block
  for (int i = tid; i < kTile * kTile; i += kThreads) {
    const int ii = i / kTile, jj = i - ii * kTile;
    const int y = y0 + ii, x = x0 + jj;
    if (y >= a.rows || x >= a.cols) continue;
    float acc = 0.0f;
    for (int t = 0; t <= 2 * rc; ++t) acc = fmaf(a.pc[t], T1[ii * UC + jj + 2 * rc - t], acc);
    const size_t o = (size_t)y * a.pitch + x;
    if (a.b) acc -= __ldg(a.b + o);
    if (a.out) a.out[o] = acc;
    if (a.partials) sq = fmaf(acc, acc, sq);
  }
  if (a.partials) {
    const double tot = block_sum<kThreads>((double)sq, red);
    if (tid == 0) a.partials[blockIdx.y * gridDim.x + blockIdx.x] = 0.5 * tot;
  }
}

// Adjoint R^* as a gather with per-sample tap orientation.
__global__ void __launch_bounds__(kThreads) k_blur_adj(const BlurArgs a) {
  pdl_entry();
  extern __shared__ float sm[];
  const int rr = a.rr, rc = a.rc;
  const int UR = kTile + 2 * rr, UC = kTile + 2 * rc;
  float* U = sm;
  float* T2 = U + UR * UC;
  int* src_c = reinterpret_cast<int*>(T2 + kTile * UC);
  unsigned char* flip_r = reinterpret_cast<unsigned char*>(src_c + UC);
  unsigned char* flip_c = flip_r + UR;
  const int y0 = blockIdx.y * kTile, x0 = blockIdx.x * kTile;
  const int tid = threadIdx.x;
  const int mode = a.bc == 3 ? 2 : a.bc;
  for (int c = tid; c < UC; c += kThreads) {
    src_c[c] = ext_src(x0 - rc + c, a.cols, mode);
    flip_c[c] = (a.bc == 1) && odd_period(x0 - rc + c, a.cols);
  }
  for (int u = tid; u < UR; u += kThreads) flip_r[u] = (a.bc == 1) && odd_period(y0 - rr + u, a.rows);
  __syncthreads();
  for (int i = tid; i < UR * UC; i += kThreads) {
    const int u = i / UC, c = i - u * UC;
    const int sr = ext_src(y0 - rr + u, a.rows, mode), sc = src_c[c];
    U[i] = (sr >= 0 && sc >= 0) ? __ldg(a.in + (size_t)sr * a.pitch + sc) : 0.0f;
  }
  __syncthreads();
  for (int i = tid; i < kTile * UC; i += kThreads) {
    const int jj = i / UC, c = i - jj * UC;
    float acc = 0.0f;
    for (int t = 0; t <= 2 * rr; ++t) {
      const float w = flip_r[jj + t] ? a.pr[2 * rr - t] : a.pr[t];
      acc = fmaf(w, U[(jj + t) * UC + c], acc);
    }
    T2[i] = acc;
  }
  __syncthreads();
  for (int i = tid; i < kTile * kTile; i += kThreads) {
    const int jj = i / kTile, cc = i - jj * kTile;
    const int y = y0 + jj, x = x0 + cc;
    if (y >= a.rows || x >= a.cols) continue;
    float acc = 0.0f;
    for (int t = 0; t <= 2 * rc; ++t) {
      const float w = flip_c[cc + t] ? a.pc[2 * rc - t] : a.pc[t];
      acc = fmaf(w, T2[jj * UC + cc + t], acc);
    }
    a.out[(size_t)y * a.pitch + x] = acc;
  }
}

// Fused g = R^*(R u - b) (+ per-CTA 1/2 ||R u - b||^2 over the CTA's own pixels).
__global__ void __launch_bounds__(kThreads) k_blur_normal(const BlurArgs a) {
  pdl_entry();
  extern __shared__ float sm[];
  const int rr = a.rr, rc = a.rc;
  const int UR = kTile + 4 * rr, UC = kTile + 4 * rc;  // u with a 2r halo
  const int VR = kTile + 2 * rr, VC = kTile + 2 * rc;  // R u - b with an r halo
  float* A = sm;                      // U (UR x UC), later V (VR x VC)
  float* B = A + UR * UC;             // T1 (VR x UC), later T2 (kTile x VC)
  int* src_c = reinterpret_cast<int*>(B + VR * UC);
  unsigned char* flip_r = reinterpret_cast<unsigned char*>(src_c + UC);
  unsigned char* flip_c = flip_r + VR;
  __shared__ double red[kThreads / 32];
  const int y0 = blockIdx.y * kTile, x0 = blockIdx.x * kTile;
  const int tid = threadIdx.x;
  const int mode = a.bc == 3 ? 2 : a.bc;
  const bool sym = a.bc == 1, per = a.bc == 3;
  for (int c = tid; c < UC; c += kThreads) src_c[c] = ext_src(x0 - 2 * rc + c, a.cols, mode);
  for (int u = tid; u < VR; u += kThreads) flip_r[u] = sym && odd_period(y0 - rr + u, a.rows);
  for (int c = tid; c < VC; c += kThreads) flip_c[c] = sym && odd_period(x0 - rc + c, a.cols);
  __syncthreads();
  for (int i = tid; i < UR * UC; i += kThreads) {
    const int u = i / UC, c = i - u * UC;
    const int sr = ext_src(y0 - 2 * rr + u, a.rows, mode), sc = src_c[c];
    A[i] = (sr >= 0 && sc >= 0) ? __ldg(a.in + (size_t)sr * a.pitch + sc) : 0.0f;
  }
  __syncthreads();
  // T1 = R along rows, on virtual rows [y0 - r, y0 + kTile + r)
  for (int i = tid; i < VR * UC; i += kThreads) {
    const int v = i / UC, c = i - v * UC;
    float acc = 0.0f;
    for (int t = 0; t <= 2 * rr; ++t) acc = fmaf(a.pr[t], A[(v + 2 * rr - t) * UC + c], acc);
    B[i] = acc;
  }
  __syncthreads();
  // V = R along columns - b, on the virtual window with an r halo
  float sq = 0.0f;  // per-thread float32 partial, float64 across the block
  for (int i = tid; i < VR * VC; i += kThreads) {
    const int v = i / VC, w = i - v * VC;
    const int y = y0 - rr + v, x = x0 - rc + w;
    const bool real = (y >= 0 && y < a.rows && x >= 0 && x < a.cols);
    float val = 0.0f;
    if (real || per) {
      float acc = 0.0f;
      for (int t = 0; t <= 2 * rc; ++t) acc = fmaf(a.pc[t], B[v * UC + w + 2 * rc - t], acc);
      if (a.b) acc -= __ldg(a.b + (size_t)pos_mod(y, a.rows) * a.pitch + pos_mod(x, a.cols));
      val = acc;
      if (a.partials && real && v >= rr && v < rr + kTile && w >= rc && w < rc + kTile) sq = fmaf(val, val, sq);
    }
    A[i] = val;
  }
  __syncthreads();
  if (sym) {  // off-image samples of the symmetric extension copy their mirror
    for (int i = tid; i < VR * VC; i += kThreads) {
      const int v = i / VC, w = i - v * VC;
      const int y = y0 - rr + v, x = x0 - rc + w;
      if (y >= 0 && y < a.rows && x >= 0 && x < a.cols) continue;
      const int sv = ext_src(y, a.rows, 1) - (y0 - rr), sw = ext_src(x, a.cols, 1) - (x0 - rc);
      float val = 0.0f;
      if (sv >= 0 && sv < VR && sw >= 0 && sw < VC) val = A[sv * VC + sw];
      A[i] = val;
    }
    __syncthreads();
  }
  // T2 = R^* along rows
  for (int i = tid; i < kTile * VC; i += kThreads) {
    const int jj = i / VC, w = i - jj * VC;
    float acc = 0.0f;
    for (int t = 0; t <= 2 * rr; ++t) {
      const float wt = flip_r[jj + t] ? a.pr[2 * rr - t] : a.pr[t];
      acc = fmaf(wt, A[(jj + t) * VC + w], acc);
    }
    B[i] = acc;
  }
  __syncthreads();
  for (int i = tid; i < kTile * kTile; i += kThreads) {
    const int jj = i / kTile, cc = i - jj * kTile;
    const int y = y0 + jj, x = x0 + cc;
    if (y >= a.rows || x >= a.cols) continue;
    float acc = 0.0f;
    for (int t = 0; t <= 2 * rc; ++t) {
      const float wt = flip_c[cc + t] ? a.pc[2 * rc - t] : a.pc[t];
      acc = fmaf(wt, B[jj * VC + cc + t], acc);
    }
    a.out[(size_t)y * a.pitch + x] = acc;
  }
  if (a.partials) {
    const double tot = block_sum<kThreads>((double)sq, red);
    if (tid == 0) a.partials[blockIdx.y * gridDim.x + blockIdx.x] = 0.5 * tot;
  }
}

void fill_args(const adjwt_blur_plan* p, BlurArgs* a) {
  *a = BlurArgs{};
  a->rows = p->rows;
  a->cols = p->cols;
  a->pitch = p->image_pitch;
  a->bc = p->bc;
  a->rr = p->kr / 2;
  a->rc = p->kc / 2;
  for (int i = 0; i < p->kr; ++i) a->pr[i] = static_cast<float>(p->taps_r[i]);
  for (int i = 0; i < p->kc; ++i) a->pc[i] = static_cast<float>(p->taps_c[i]);
}

dim3 grid_of(const adjwt_blur_plan* p) {
  return dim3((p->cols + kTile - 1) / kTile, (p->rows + kTile - 1) / kTile);
}

size_t smem_fwd(int rr, int rc) {
  const int UR = kTile + 2 * rr, UC = kTile + 2 * rc;
  return (size_t)(UR * UC + kTile * UC) * 4 + UC * 4 + UR + UC + 16;
}
size_t smem_normal(int rr, int rc) {
  const int UR = kTile + 4 * rr, UC = kTile + 4 * rc, VR = kTile + 2 * rr, VC = kTile + 2 * rc;
  return (size_t)(UR * UC + VR * UC) * 4 + UC * 4 + VR + VC + 16;
}

template <typename K>
int launch(const char* name, K kernel, const adjwt_blur_plan* p, const BlurArgs& a, size_t smem, cudaStream_t s) {
  if (smem > 48 * 1024) ADJWT_CUDA_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                             static_cast<int>(smem)));
  ADJWT_TRACED(name, 0, s, pdl_launch(kernel, grid_of(p), kThreads, smem, s, a));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  return ADJWT_OK;
}

}  // namespace

int blur_partial_slots(const adjwt_blur_plan* p) {
  dim3 g = grid_of(p);
  int slots = static_cast<int>(g.x * g.y);
  if (tiled_blur_supported(p)) slots = std::max(slots, tiled_blur_grid_slots(p));
  if (tma_blur_supported(p)) slots = std::max(slots, tma_blur_partial_slots(p));
  return slots;
}

int launch_blur(const adjwt_blur_plan* p, const float* in, float* out, bool adjoint, cudaStream_t s) {
  if (tma_blur_supported(p)) return launch_tma_blur(p, adjoint, in, nullptr, out, nullptr, s, nullptr);
  BlurArgs a;
  fill_args(p, &a);
  a.in = in;
  a.out = out;
  const size_t smem = smem_fwd(a.rr, a.rc);
  return adjoint ? launch("blur_adjoint", k_blur_adj, p, a, smem, s) : launch("blur", k_blur_fwd, p, a, smem, s);
}

int launch_blur_normal(const adjwt_blur_plan* p, const float* u, const float* b, float* g, double* partials,
                       float* scratch_v, cudaStream_t s, int* nparts) {
  if (scratch_v && tma_blur_supported(p)) {  // v = R u - b, then g = R^* v
    int rc = launch_tma_blur(p, false, u, b, scratch_v, partials, s, nparts);
    if (rc) return rc;
    return launch_tma_blur(p, true, scratch_v, nullptr, g, nullptr, s, nullptr);
  }
  if (tiled_blur_supported(p)) {
    if (nparts) *nparts = tiled_blur_grid_slots(p);
    return launch_tiled_blur(p, u, b, g, partials, s);
  }
  if (nparts) *nparts = static_cast<int>(grid_of(p).x * grid_of(p).y);
  BlurArgs a;
  fill_args(p, &a);
  a.in = u;
  a.b = b;
  a.out = g;
  a.partials = partials;
  return launch("blur_normal", k_blur_normal, p, a, smem_normal(a.rr, a.rc), s);
}

int launch_blur_residual_norm(const adjwt_blur_plan* p, const float* u, const float* b, double* partials,
                              cudaStream_t s, int* nparts) {
  if (tma_blur_supported(p)) return launch_tma_blur(p, false, u, b, nullptr, partials, s, nparts);
  if (nparts) *nparts = static_cast<int>(grid_of(p).x * grid_of(p).y);
  BlurArgs a;
  fill_args(p, &a);
  a.in = u;
  a.b = b;
  a.out = nullptr;
  a.partials = partials;
  return launch("blur_residual", k_blur_fwd, p, a, smem_fwd(a.rr, a.rc), s);
}

}  // namespace adjwt
