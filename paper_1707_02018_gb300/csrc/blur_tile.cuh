// Tiled body of the fused blur normal operator g = R^*(R u - b) (Sec. I,
// the gradient after Eq. 1), one kT x kT output tile per call, for PSF radii
// up to kTiledMaxRadius (compile-time radius; the shorter axis is zero-padded
// to the same radius, which leaves the operator unchanged).  Shared by the
// fused blur kernel (blur_tiled.cu) and the batched FISTA engine
// (fista_batch.cu).
//
// Same operator definitions as blur_kernels.cu.  The tile runs the separable
// passes in shared memory.  Every pass is a 1D correlation executed by threads
// that each produce kRB consecutive outputs along the filter direction from
// one sliding window held in registers (kRB + 2R shared-memory loads for
// kRB * (2R + 1) FMAs):
//   vertical passes:   lanes take consecutive columns (conflict-free rows),
//   horizontal passes: lanes take consecutive rows (odd row pitches keep the
//                      32 lanes on 32 banks).
// The boundary extension is applied when the tile is gathered from global
// memory; tiles that touch the border of a symmetric image switch to the
// orientation-aware taps of R^* (see blur_kernels.cu) and refill the
// off-image samples of R u - b from their mirror.
#pragma once

#include "adjwt_internal.h"
#include "device_common.cuh"

namespace adjwt {
namespace {

constexpr int kTiledMaxRadius = 12;

constexpr int kT = 64;        // output tile side
constexpr int kRB = 16;       // outputs per thread per pass
constexpr int kNT = 256;      // threads per CTA

__host__ __device__ constexpr int odd_up(int v) { return v | 1; }
__host__ __device__ constexpr int ceil_to(int v, int m) { return (v + m - 1) / m * m; }

template <int R>
struct Geo {
  // fused kernel
  static constexpr int VR = kT + 2 * R;                    // rows of R u - b
  static constexpr int VC = kT + 2 * R;
  static constexpr int UR = ceil_to(VR, kRB) + 2 * R;      // rows read by pass 1
  static constexpr int UC = kT + 4 * R;
  static constexpr int UP = odd_up(UC);
  static constexpr int T1R = VR;
  static constexpr int T1P = odd_up(ceil_to(VC, kRB) + 2 * R);  // cols read by pass 2
  static constexpr int VP = odd_up(ceil_to(VC, kRB));
  static constexpr int VROWS = ceil_to(kT, kRB) + 2 * R;   // rows read by pass 3
  static constexpr int T2P = odd_up(ceil_to(kT, kRB) + 2 * R);
  static constexpr int A_FLOATS = (UR * UP > VROWS * VP) ? UR * UP : VROWS * VP;
  static constexpr int B_FLOATS = (T1R * T1P > kT * T2P) ? T1R * T1P : kT * T2P;
};

struct TiledArgs {
  const float* in;
  const float* b;
  float* out;
  double* partials;
  int rows, cols, pitch, bc;  // bc: 0 zero, 1 sym, 3 per
  int* status;  // device status word (checked builds record ADJWT_ERR_BOUNDS here)
  float pr[2 * kTiledMaxRadius + 1], pc[2 * kTiledMaxRadius + 1];  // padded to 2R+1
};

__device__ __forceinline__ bool odd_period(int x, int N) { return (floor_div(x, N) & 1) != 0; }

// out[i][c] = sum_t w[t] in[i + t][c], i in [0, nrows), c in [0, ncols)
template <int R, bool FLIP>
__device__ __forceinline__ void vpass(const float* __restrict__ in, int in_p, float* __restrict__ out, int out_p,
                                      int nrows, int ncols, const float (&w)[2 * R + 1],
                                      const unsigned char* __restrict__ flip) {
  constexpr int K = 2 * R + 1;
  const int nblk = (nrows + kRB - 1) / kRB;
  for (int item = threadIdx.x; item < nblk * ncols; item += kNT) {
    const int blk = item / ncols, c = item - blk * ncols;
    const int i0 = blk * kRB;
    float acc[kRB];
#pragma unroll
    for (int o = 0; o < kRB; ++o) acc[o] = 0.0f;
#pragma unroll
    for (int j = 0; j < kRB + 2 * R; ++j) {
      const float v = in[(i0 + j) * in_p + c];
      bool f = false;
      if (FLIP) f = flip[i0 + j];
#pragma unroll
      for (int o = 0; o < kRB; ++o) {
        const int t = j - o;
        if (t >= 0 && t < K) acc[o] = fmaf(FLIP ? (f ? w[K - 1 - t] : w[t]) : w[t], v, acc[o]);
      }
    }
#pragma unroll
    for (int o = 0; o < kRB; ++o)
      if (i0 + o < nrows) out[(i0 + o) * out_p + c] = acc[o];
  }
}

// out[r][i] = sum_t w[t] in[r][i + t] (- bsub[r][i]); r in [0, nrows), i in [0, ncols)
template <int R, bool FLIP>
__device__ __forceinline__ void hpass(const float* __restrict__ in, int in_p, float* __restrict__ out, int out_p,
                                      int nrows, int ncols, const float (&w)[2 * R + 1],
                                      const unsigned char* __restrict__ flip) {
  constexpr int K = 2 * R + 1;
  const int nblk = (ncols + kRB - 1) / kRB;
  for (int item = threadIdx.x; item < nblk * nrows; item += kNT) {
    const int blk = item / nrows, r = item - blk * nrows;
    const int i0 = blk * kRB;
    float acc[kRB];
#pragma unroll
    for (int o = 0; o < kRB; ++o) acc[o] = 0.0f;
#pragma unroll
    for (int j = 0; j < kRB + 2 * R; ++j) {
      const float v = in[r * in_p + i0 + j];
      bool f = false;
      if (FLIP) f = flip[i0 + j];
#pragma unroll
      for (int o = 0; o < kRB; ++o) {
        const int t = j - o;
        if (t >= 0 && t < K) acc[o] = fmaf(FLIP ? (f ? w[K - 1 - t] : w[t]) : w[t], v, acc[o]);
      }
    }
#pragma unroll
    for (int o = 0; o < kRB; ++o)
      if (i0 + o < ncols) out[r * out_p + i0 + o] = acc[o];
  }
}

// Final horizontal pass straight to global memory (kRB outputs -> kRB/4 float4).
template <int R, bool FLIP>
__device__ __forceinline__ void hpass_store(const float* __restrict__ in, int in_p, const TiledArgs& a, int y0,
                                            int x0, const float (&w)[2 * R + 1],
                                            const unsigned char* __restrict__ flip, const float* __restrict__ bsub,
                                            float* sq) {
  constexpr int K = 2 * R + 1;
  constexpr int nblk = kT / kRB;
  for (int item = threadIdx.x; item < nblk * kT; item += kNT) {
    const int blk = item / kT, r = item - blk * kT;
    const int i0 = blk * kRB;
    const int y = y0 + r;
    if (y >= a.rows) continue;
    float acc[kRB];
#pragma unroll
    for (int o = 0; o < kRB; ++o) acc[o] = 0.0f;
#pragma unroll
    for (int j = 0; j < kRB + 2 * R; ++j) {
      const float v = in[r * in_p + i0 + j];
      bool f = false;
      if (FLIP) f = flip[i0 + j];
#pragma unroll
      for (int o = 0; o < kRB; ++o) {
        const int t = j - o;
        if (t >= 0 && t < K) acc[o] = fmaf(FLIP ? (f ? w[K - 1 - t] : w[t]) : w[t], v, acc[o]);
      }
    }
    const int x = x0 + i0;
    if (x >= a.cols) continue;  // a block past the last column of the last tile: nothing to store
    if (!in_bounds(a.status, y >= 0 && x >= 0 && x < a.pitch)) continue;
    float* dst = a.out ? a.out + (size_t)y * a.pitch + x : nullptr;
    const float* bb = bsub ? bsub + (size_t)y * a.pitch + x : nullptr;
    if (x + kRB <= a.cols) {
      if (bb) {
#pragma unroll
        for (int q = 0; q < kRB / 4; ++q) {
          const float4 b4 = __ldg(reinterpret_cast<const float4*>(bb) + q);
          acc[4 * q] -= b4.x;
          acc[4 * q + 1] -= b4.y;
          acc[4 * q + 2] -= b4.z;
          acc[4 * q + 3] -= b4.w;
        }
      }
      if (sq) {
#pragma unroll
        for (int o = 0; o < kRB; ++o) *sq = fmaf(acc[o], acc[o], *sq);
      }
      if (dst) {
#pragma unroll
        for (int q = 0; q < kRB / 4; ++q)
          reinterpret_cast<float4*>(dst)[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
      }
    } else {
#pragma unroll
      for (int o = 0; o < kRB; ++o) {
        if (x + o < a.cols) {
          float v = acc[o];
          if (bb) v -= __ldg(bb + o);
          if (sq) *sq = fmaf(v, v, *sq);
          if (dst) dst[o] = v;
        }
      }
    }
  }
}

template <int R>
__device__ __forceinline__ void load_taps(const TiledArgs& a, float (&pr)[2 * R + 1], float (&pc)[2 * R + 1],
                                          bool reversed) {
#pragma unroll
  for (int t = 0; t < 2 * R + 1; ++t) {
    pr[t] = reversed ? a.pr[2 * R - t] : a.pr[t];
    pc[t] = reversed ? a.pc[2 * R - t] : a.pc[t];
  }
}

// Gather rows [oy, oy + NR) x cols [ox, ox + NC) of the boundary-extended
// image into smem (pitch sp).  Each thread keeps 16 independent loads in
// flight; a window that lies inside the image skips the extension map.
template <int NR, int NC, bool CG = false>
__device__ __forceinline__ void gather(const float* __restrict__ img, int rows, int cols, int pitch, int mode,
                                       int oy, int ox, float* __restrict__ dst, int sp,
                                       const int* __restrict__ src_c, int* status = nullptr) {
  constexpr int total = NR * NC;
  constexpr int U = 16;
  const bool inside = oy >= 0 && ox >= 0 && oy + NR <= rows && ox + NC <= cols;
  const float* base = img + (size_t)(inside ? oy : 0) * pitch + (inside ? ox : 0);
  for (int b0 = threadIdx.x; b0 < total; b0 += U * kNT) {
    float v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = b0 + u * kNT;
      v[u] = 0.0f;
      if (i < total) {
        const int rr = i / NC, cc = i - rr * NC;
        if (inside) {
          if (in_bounds(status, oy + rr < rows && ox + cc < cols))
            v[u] = CG ? __ldcg(base + (size_t)rr * pitch + cc) : __ldg(base + (size_t)rr * pitch + cc);
        } else {
          const int sr = ext_src(oy + rr, rows, mode), sc = src_c[cc];
          if (sr >= 0 && sc >= 0 && in_bounds(status, sr < rows && sc < cols))
            v[u] = CG ? __ldcg(img + (size_t)sr * pitch + sc) : __ldg(img + (size_t)sr * pitch + sc);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = b0 + u * kNT;
      if (i < total) {
        const int rr = i / NC, cc = i - rr * NC;
        dst[rr * sp + cc] = v[u];
      }
    }
  }
}

// One kT x kT tile (tile_y, tile_x) of g = R^*(R u - b); adds this thread's
// float32 partial of (R u - b)^2 over the tile's own pixels to sq.  sm: the
// caller's blur_tile_smem<R>() bytes of shared memory; NT = kNT threads.
// CG: u was written earlier in the same launch (read at L2).
template <int R, bool CG = false>
__device__ __forceinline__ void blur_normal_tile(const TiledArgs& a, int tile_y, int tile_x, float* sm, int* s_border_,
                                                 float& sq) {
  using G = Geo<R>;
  float* A = sm;
  float* B = A + G::A_FLOATS;
  int* src_c = reinterpret_cast<int*>(B + G::B_FLOATS);
  unsigned char* flip_r = reinterpret_cast<unsigned char*>(src_c + G::UC);
  unsigned char* flip_c = flip_r + G::VROWS;
  int& s_border = *s_border_;
  const int y0 = tile_y * kT, x0 = tile_x * kT;
  const int tid = threadIdx.x;
  const int mode = a.bc == 3 ? 2 : a.bc;
  const bool sym = a.bc == 1, per = a.bc == 3;
  // does the R u - b window leave the image?  (then SYM flips / ZERO zeros apply)
  const bool border = (y0 - R < 0) || (x0 - R < 0) || (y0 + kT + R > a.rows) || (x0 + kT + R > a.cols);
  if (tid == 0) s_border = border;
  for (int c = tid; c < G::UC; c += kNT) src_c[c] = ext_src(x0 - 2 * R + c, a.cols, mode);
  for (int u = tid; u < G::VROWS; u += kNT) flip_r[u] = sym && odd_period(y0 - R + u, a.rows);
  for (int c = tid; c < G::VP; c += kNT) flip_c[c] = sym && odd_period(x0 - R + c, a.cols);
  __syncthreads();
  gather<G::UR, G::UC, CG>(a.in, a.rows, a.cols, a.pitch, mode, y0 - 2 * R, x0 - 2 * R, A, G::UP, src_c, a.status);
  __syncthreads();
  float pr[2 * R + 1], pc[2 * R + 1];
  load_taps<R>(a, pr, pc, true);  // convolution = correlation with reversed taps
  vpass<R, false>(A, G::UP, B, G::T1P, G::VR, G::UC, pr, nullptr);
  __syncthreads();
  hpass<R, false>(B, G::T1P, A, G::VP, G::VR, G::VC, pc, nullptr);
  __syncthreads();
  // subtract b and fix the off-image samples (sq: per-thread float32 partial)
  {
    constexpr int total = G::VR * G::VC, U = 16;
    for (int b0 = tid; b0 < total; b0 += U * kNT) {
      float bv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {  // all b loads of this round in flight first
        const int i = b0 + u * kNT;
        bv[u] = 0.0f;
        if (i < total && a.b) {
          const int v = i / G::VC, w = i - v * G::VC;
          const int y = y0 - R + v, x = x0 - R + w;
          const bool real = y >= 0 && y < a.rows && x >= 0 && x < a.cols;
          if (real) {
            bv[u] = __ldg(a.b + (size_t)y * a.pitch + x);
          } else if (per) {
            bv[u] = __ldg(a.b + (size_t)pos_mod(y, a.rows) * a.pitch + pos_mod(x, a.cols));
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = b0 + u * kNT;
        if (i >= total) break;
        const int v = i / G::VC, w = i - v * G::VC;
        const int y = y0 - R + v, x = x0 - R + w;
        const bool real = y >= 0 && y < a.rows && x >= 0 && x < a.cols;
        float val = A[v * G::VP + w];
        if (real || per) {
          val -= bv[u];
          if (a.partials && real && v >= R && v < R + kT && w >= R && w < R + kT) sq = fmaf(val, val, sq);
        } else {
          val = 0.0f;
        }
        A[v * G::VP + w] = val;
      }
    }
  }
  __syncthreads();
  if (sym && s_border) {
    for (int i = tid; i < G::VR * G::VC; i += kNT) {
      const int v = i / G::VC, w = i - v * G::VC;
      const int y = y0 - R + v, x = x0 - R + w;
      if (y >= 0 && y < a.rows && x >= 0 && x < a.cols) continue;
      const int sv = ext_src(y, a.rows, 1) - (y0 - R), sw = ext_src(x, a.cols, 1) - (x0 - R);
      float val = 0.0f;
      if (sv >= 0 && sv < G::VR && sw >= 0 && sw < G::VC) val = A[sv * G::VP + sw];
      A[v * G::VP + w] = val;
    }
    __syncthreads();
  }
  load_taps<R>(a, pr, pc, false);  // adjoint = correlation with the taps as given
  if (sym && s_border) {
    vpass<R, true>(A, G::VP, B, G::T2P, kT, G::VC, pr, flip_r);
    __syncthreads();
    hpass_store<R, true>(B, G::T2P, a, y0, x0, pc, flip_c, nullptr, nullptr);
  } else {
    vpass<R, false>(A, G::VP, B, G::T2P, kT, G::VC, pr, nullptr);
    __syncthreads();
    hpass_store<R, false>(B, G::T2P, a, y0, x0, pc, nullptr, nullptr, nullptr);
  }
}

template <int R>
constexpr size_t blur_tile_smem() {
  using G = Geo<R>;
  return (size_t)(G::A_FLOATS + G::B_FLOATS) * 4 + G::UC * 4 + G::VROWS + G::VP + 16;
}


}  // namespace
}  // namespace adjwt
