// One kWH x kWW output tile of the gradient of the data term (Sec. I, after
// Eq. 1), g = R^*(R u - b), from TMA-staged windows: the batched FISTA
// engine's blur stage (fista_batch.cu), for problems whose R^* needs no
// orientation-aware taps (zero or periodic boundaries, or palindromic taps).
//
// The TMA unit copies the (kWH + 4R) x (kWW + 2 XU) window of u and the
// (kWH + 2R) x (kWW + 2 XB) window of b (XB = R, XU = XB + R, both rounded up
// to 4 floats so that the boxes start 16-byte aligned; the copies' zero fill
// is the zero extension).  Off-image cells under the symmetric and periodic
// extensions are then completed by the threads.  Four separable passes run in
// shared memory:
//   A  vertical R on the u window                -> T1   (kWH + 2R rows)
//   B  horizontal R on T1                        -> R u over the residual window
//   C  vertical R^* on (R u - b)                 -> T2   (kWH rows)
//   D  horizontal R^* on T2                      -> g (staged, then row stores)
// The residual window is the region R^* reads: its off-image cells take the
// extension of r = R u - b (zero: 0; periodic: R u and b of the wrapped cell,
// computed directly from the wrapped u and b windows; half-point symmetric:
// copied from the mirror cell inside the window, exact for palindromic taps).
// R u is kept in the u buffer pass A has consumed, T2 in T1, the output tile
// in the u buffer again.  Every pass is a register-window 1D correlation:
// 16 (pass D: 8) consecutive outputs a thread from 16 + 2R loads.
#pragma once

#include "adjwt_internal.h"
#include "blur_tile.cuh"
#include "device_common.cuh"
#include "tma.cuh"

namespace adjwt {
namespace {

constexpr int kWH = 32;  // output rows of a window tile
constexpr int kWW = 64;  // output columns
constexpr int kWT = 256; // threads

__host__ __device__ constexpr int win_up4(int v) { return (v + 3) / 4 * 4; }
__host__ __device__ constexpr int win_up32(int v) { return (v + 31) / 32 * 32; }

template <int R>
struct WG {
  static constexpr int K = 2 * R + 1;
  static constexpr int XB = win_up4(R);            // residual / b window columns left of the tile
  static constexpr int XU = win_up4(XB + R);       // u window columns left of the tile
  static constexpr int DU = XU - XB - R;           // T1 column c is u window column c + DU
  static constexpr int UH = kWH + 4 * R;           // u window (TMA box)
  static constexpr int UW = kWW + 2 * XU;
  static constexpr int VH = kWH + 2 * R;           // residual / b window (TMA box for b)
  static constexpr int VW = kWW + 2 * XB;
  static constexpr int T1W = VW + 2 * R;           // columns of pass A
  static constexpr int T1P = T1W | 1;              // odd pitches: row-wise passes put lanes on rows
  static constexpr int VP = VW | 1;
  static constexpr int T2P = VW | 1;
  static constexpr int StP = kWW + 4;              // output staging: a quarter warp's 16-byte stores on distinct banks
  static constexpr int UBUF = win_up32(UH * UW);
  static constexpr int BBUF = win_up32(VH * VW);
  static constexpr int T1BUF = win_up32(VH * T1P);
  static_assert(VH >= 16 && VW >= 16, "passes work in blocks of 16");
  static_assert(VH * VP <= UBUF && kWH * StP <= UBUF, "R u and the output tile fit in the u buffer");
  static_assert(kWH * T2P <= T1BUF, "T2 fits in T1");
  // buffers, then the mbarrier (8-byte aligned: the buffers are 128-byte multiples)
  static constexpr size_t smem_bytes() { return (size_t)(UBUF + BBUF + T1BUF) * 4 + 16; }
};

// Box dimensions of WG<R> for a runtime radius (host: the tensor maps).
inline void window_boxes(int R, int* uh, int* uw, int* vh, int* vw) {
  const int xb = win_up4(R), xu = win_up4(xb + R);
  *uh = kWH + 4 * R;
  *uw = kWW + 2 * xu;
  *vh = kWH + 2 * R;
  *vw = kWW + 2 * xb;
}

// Source of virtual index x under the symmetric (1) / periodic (2) extension.
__device__ __forceinline__ int win_ext(int x, int N, int mode) {
  if (x >= 0 && x < N) return x;
  if (x >= -N && x < 2 * N) {
    if (mode == 1) return x < 0 ? -1 - x : 2 * N - 1 - x;
    return x < 0 ? x + N : x - N;
  }
  return ext_src(x, N, mode);
}

// Off-image cells of a BH x BW box whose top-left cell is image (oy, ox):
// rows above / below the image (full width), then the columns left / right
// of it on the other rows.
template <int BH, int BW>
struct WinStrips {
  int oy, ox, rlo, rhi, clo, chi, side, ntop, nbot, total;
  __device__ __forceinline__ WinStrips(int rows, int cols, int oy_, int ox_) : oy(oy_), ox(ox_) {
    rlo = min(max(-oy, 0), BH);
    rhi = min(max(rows - oy, rlo), BH);
    clo = min(max(-ox, 0), BW);
    chi = min(max(cols - ox, clo), BW);
    side = clo + (BW - chi);
    ntop = rlo * BW;
    nbot = (BH - rhi) * BW;
    total = ntop + nbot + (rhi - rlo) * side;
  }
  __device__ __forceinline__ int cell(int i) const {
    if (i < ntop) return i;
    if (i < ntop + nbot) return rhi * BW + (i - ntop);
    const int j = i - ntop - nbot, rr = j / side, k = j - rr * side;
    return (rlo + rr) * BW + (k < clo ? k : chi + (k - clo));
  }
  // the extended image at box cell c (read at L2: u is written in the same launch)
  __device__ __forceinline__ float load(const float* img, int rows, int cols, int pitch, int mode, int* status,
                                        int c) const {
    const int rr = c / BW, cc = c - rr * BW;
    const int sr = win_ext(oy + rr, rows, mode), sc = win_ext(ox + cc, cols, mode);
    if (!in_bounds(status, sr >= 0 && sr < rows && sc >= 0 && sc < cols)) return 0.0f;
    return __ldcg(img + (size_t)sr * pitch + sc);
  }
};

constexpr int kWinFill = 8;  // off-image cells per thread fetched before the copies land

// Tile (ty, tx) of g = R^*(R u - b); returns this thread's float32 partial of
// (R u - b)^2 over the tile's own pixels (when a.partials is set).  umap / bmap:
// tensor maps over u and b with the WG<R> boxes (in device memory).  dyn:
// WG<R>::smem_bytes() of 128-byte aligned shared memory.  A copy that does
// not land within the bounded wait records ADJWT_ERR_TIMEOUT (the tile is then
// not written).
template <int R>
__device__ __forceinline__ float blur_window_tile(const TiledArgs& a, const CUtensorMap* umap,
                                                  const CUtensorMap* bmap, int ty, int tx, unsigned char* dyn) {
  using G = WG<R>;
  constexpr int K = G::K;
  float* const U = reinterpret_cast<float*>(dyn);
  float* const Bw = U + G::UBUF;
  float* const T1 = Bw + G::BBUF;
  float* const T2 = T1;
  float* const Ru = U;
  float* const St = U;
  uint64_t* const bar = reinterpret_cast<uint64_t*>(T1 + G::T1BUF);
  const int tid = threadIdx.x;
  const int y0 = ty * kWH, x0 = tx * kWW;
  const int mode = a.bc == 3 ? 2 : a.bc;
  const bool has_b = a.b != nullptr;
  // R is a convolution (reversed taps), R^* a correlation (taps as given)
  float pr[K], pc[K];
#pragma unroll
  for (int t = 0; t < K; ++t) {
    pr[t] = a.pr[t];
    pc[t] = a.pc[t];
  }

  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    // the buffers' earlier generic-proxy use (other stage bodies) comes before
    // the copies' writes; u was written earlier in this launch by other CTAs
    // (generic stores, published with a release this thread has acquired):
    // those writes come before the copies' reads
    fence_proxy_async();
    asm volatile("fence.proxy.async.global;" ::: "memory");
    mbar_arrive_expect_tx(bar, (uint32_t)(G::UH * G::UW + (has_b ? G::VH * G::VW : 0)) * 4u);
    tma_load_2d(U, umap, bar, x0 - G::XU, y0 - 2 * R);
    if (has_b) tma_load_2d(Bw, bmap, bar, x0 - G::XB, y0 - R);
  }
  // off-image cells: fetched through the extension map while the copies are in flight
  const bool uedge = y0 - 2 * R < 0 || x0 - G::XU < 0 || y0 + kWH + 2 * R > a.rows || x0 + kWW + G::XU > a.cols;
  const bool redge = y0 - R < 0 || x0 - G::XB < 0 || y0 + kWH + R > a.rows || x0 + kWW + G::XB > a.cols;
  const bool fill_u = uedge && mode != 0;
  const bool fill_b = redge && mode == 2 && has_b;
  const WinStrips<G::UH, G::UW> su(a.rows, a.cols, y0 - 2 * R, x0 - G::XU);
  const WinStrips<G::VH, G::VW> sb(a.rows, a.cols, y0 - R, x0 - G::XB);
  float fu[kWinFill];
  if (fill_u) {
#pragma unroll
    for (int q = 0; q < kWinFill; ++q) {
      const int i = tid + q * kWT;
      fu[q] = i < su.total ? su.load(a.in, a.rows, a.cols, a.pitch, mode, a.status, su.cell(i)) : 0.0f;
    }
  }
  __syncthreads();  // the barrier's initialisation is visible
  const bool ok = mbar_wait(bar, 0);
  if (!__syncthreads_and(ok)) {
    if (tid == 0) {
      record_status(a.status, ADJWT_ERR_TIMEOUT);
      (void)mbar_wait(bar, 0);  // one more bounded wait before the buffers are reused
    }
    __syncthreads();
    return 0.0f;
  }
  if (fill_u || fill_b) {
    if (fill_u) {
#pragma unroll
      for (int q = 0; q < kWinFill; ++q) {
        const int i = tid + q * kWT;
        if (i < su.total) U[su.cell(i)] = fu[q];
      }
      for (int i = tid + kWinFill * kWT; i < su.total; i += kWT) {  // large overhangs (small images)
        const int c = su.cell(i);
        U[c] = su.load(a.in, a.rows, a.cols, a.pitch, mode, a.status, c);
      }
    }
    if (fill_b) {
      for (int i = tid; i < sb.total; i += kWT) {
        const int c = sb.cell(i), rr = c / G::VW, cc = c - rr * G::VW;
        const int sr = win_ext(y0 - R + rr, a.rows, 2), sc = win_ext(x0 - G::XB + cc, a.cols, 2);
        Bw[c] = in_bounds(a.status, sr >= 0 && sr < a.rows && sc >= 0 && sc < a.cols)
                    ? __ldg(a.b + (size_t)sr * a.pitch + sc)
                    : 0.0f;
      }
    }
    __syncthreads();
  }

  // A: T1[r][c] = sum_t q[t] U[r + t][c + DU] (q: taps reversed), 16 rows of
  //    one column a thread, lanes on consecutive columns
  {
    constexpr int NA = (G::VH + 15) / 16;
    for (int item = tid; item < NA * G::T1W; item += kWT) {
      const int blk = item / G::T1W, c = item - blk * G::T1W;
      const int s = min(16 * blk, G::VH - 16);  // the last block overlaps its neighbour
      const float* src = U + s * G::UW + c + G::DU;
      float acc[16];
#pragma unroll
      for (int o = 0; o < 16; ++o) acc[o] = 0.0f;
#pragma unroll
      for (int j = 0; j < 16 + 2 * R; ++j) {
        const float v = src[j * G::UW];
#pragma unroll
        for (int o = 0; o < 16; ++o) {
          const int t = j - o;
          if (t >= 0 && t < K) acc[o] = fmaf(pr[K - 1 - t], v, acc[o]);
        }
      }
      float* dst = T1 + s * G::T1P + c;
#pragma unroll
      for (int o = 0; o < 16; ++o) dst[o * G::T1P] = acc[o];
    }
  }
  __syncthreads();

  // B: R u over the residual window, 16 consecutive columns of one row a
  //    thread; a half warp takes 16 consecutive rows of one column block (the
  //    two halves of a warp on disjoint bank ranges); zero extension: R u - b
  //    vanishes off the image
  {
    constexpr int NB = (G::VW + 15) / 16, NG = (G::VH + 15) / 16;
    for (int h = tid >> 4; h < NB * NG; h += kWT / 16) {
      const int blk = h / NG, r = 16 * (h - blk * NG) + (tid & 15);
      if (r >= G::VH) continue;
      const int s = min(16 * blk, G::VW - 16);
      const float* src = T1 + r * G::T1P + s;
      float acc[16];
#pragma unroll
      for (int o = 0; o < 16; ++o) acc[o] = 0.0f;
#pragma unroll
      for (int j = 0; j < 16 + 2 * R; ++j) {
        const float v = src[j];
#pragma unroll
        for (int o = 0; o < 16; ++o) {
          const int t = j - o;
          if (t >= 0 && t < K) acc[o] = fmaf(pc[K - 1 - t], v, acc[o]);
        }
      }
      if (mode == 0 && redge) {
        const int y = y0 - R + r;
#pragma unroll
        for (int o = 0; o < 16; ++o) {
          const int x = x0 - G::XB + s + o;
          if (y < 0 || y >= a.rows || x < 0 || x >= a.cols) acc[o] = 0.0f;
        }
      }
      float* dst = Ru + r * G::VP + s;
#pragma unroll
      for (int o = 0; o < 16; ++o) dst[o] = acc[o];
    }
  }
  __syncthreads();

  // half-point symmetric extension of r = R u - b: off-image cells of the
  // residual window take the value of their mirror cell (inside the window)
  if (mode == 1 && redge) {
    for (int i = tid; i < sb.total; i += kWT) {
      const int c = sb.cell(i), rr = c / G::VW, cc = c - rr * G::VW;
      const int my = ext_src(y0 - R + rr, a.rows, 1) - (y0 - R);
      const int mx = ext_src(x0 - G::XB + cc, a.cols, 1) - (x0 - G::XB);
      const bool in = my >= 0 && my < G::VH && mx >= 0 && mx < G::VW;
      Ru[rr * G::VP + cc] = in ? Ru[my * G::VP + mx] : 0.0f;
      if (has_b) Bw[rr * G::VW + cc] = in ? Bw[my * G::VW + mx] : 0.0f;
    }
    __syncthreads();
  }

  // C: T2[r][c] = sum_t p[t] (R u - b)[r + t][c] (correlation), 16 rows of
  //    one column a thread, lanes on consecutive columns; the tile's own
  //    pixels add to the float32 partial of (R u - b)^2
  float sq = 0.0f;
  {
    for (int item = tid; item < 2 * G::VW; item += kWT) {
      const int blk = item / G::VW, c = item - blk * G::VW;
      const int s = 16 * blk;
      const float* src = Ru + s * G::VP + c;
      const float* bsrc = Bw + s * G::VW + c;
      const bool own_c = a.partials != nullptr && c >= G::XB && c < G::XB + kWW && x0 - G::XB + c < a.cols;
      float acc[16];
#pragma unroll
      for (int o = 0; o < 16; ++o) acc[o] = 0.0f;
#pragma unroll
      for (int j = 0; j < 16 + 2 * R; ++j) {
        float v = src[j * G::VP];
        if (has_b) v -= bsrc[j * G::VW];
        if (j >= R && j < R + 16) {
          if (own_c && y0 + s + (j - R) < a.rows) sq = fmaf(v, v, sq);
        }
#pragma unroll
        for (int o = 0; o < 16; ++o) {
          const int t = j - o;
          if (t >= 0 && t < K) acc[o] = fmaf(pr[t], v, acc[o]);
        }
      }
      float* dst = T2 + s * G::T2P + c;
#pragma unroll
      for (int o = 0; o < 16; ++o) dst[o * G::T2P] = acc[o];
    }
  }
  __syncthreads();

  // D: g[y0 + r][x0 + x] = sum_t p[t] T2[r][x + XB - R + t], 8 consecutive
  //    outputs of one row a thread (lanes on rows) into a staging tile, then
  //    each warp stores whole rows
  if (a.out) {
    for (int item = tid; item < (kWW / 8) * kWH; item += kWT) {
      const int blk = item / kWH, r = item - blk * kWH;
      const int s = 8 * blk;
      const float* src = T2 + r * G::T2P + s + G::XB - R;
      float acc[8];
#pragma unroll
      for (int o = 0; o < 8; ++o) acc[o] = 0.0f;
#pragma unroll
      for (int j = 0; j < 8 + 2 * R; ++j) {
        const float v = src[j];
#pragma unroll
        for (int o = 0; o < 8; ++o) {
          const int t = j - o;
          if (t >= 0 && t < K) acc[o] = fmaf(pc[t], v, acc[o]);
        }
      }
      float4* st = reinterpret_cast<float4*>(St + r * G::StP + s);
      st[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
      st[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
    }
    __syncthreads();
    for (int i = tid; i < kWH * (kWW / 4); i += kWT) {
      const int r = i / (kWW / 4), c4 = 4 * (i - r * (kWW / 4));
      const int y = y0 + r, x = x0 + c4;
      if (y >= a.rows || x >= a.cols || !in_bounds(a.status, x < a.pitch)) continue;
      const float4 v = *reinterpret_cast<const float4*>(St + r * G::StP + c4);
      float* dst = a.out + (size_t)y * a.pitch + x;
      if (x + 4 <= a.cols) {
        *reinterpret_cast<float4*>(dst) = v;
      } else {
        const float e[4] = {v.x, v.y, v.z, v.w};
        for (int q = 0; q < 4 && x + q < a.cols; ++q) dst[q] = e[q];
      }
    }
  }
  __syncthreads();
  if (tid == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
  return sq;
}

}  // namespace
}  // namespace adjwt
