// Multi-level 2D wavelet kernels: W (reconstruction), W^* (exact adjoint,
// Eq. 4) and W^dagger (analysis), one launch per level.
//
// Analysis direction (W^* and W^dagger), one level, per axis:
//     out[k] = sum_i f[i] z[2k+1-i],   z[e] = w(e) * y[src(e)]
// with e the coordinate of the length N + 2L' extended signal, src(e) the
// extension map of Sec. I-A (zero / half-point symmetric / periodic) and
// w = 1/c for W^* (the weighted extension (E^dagger)^*, Eq. 2) or 1 for
// W^dagger; f are the dual analysis filters (reversed synthesis filters,
// Eq. 3 / Eq. 4) for W^* and the analysis filters for W^dagger.  The
// extension is applied in the load path: each CTA gathers its extended tile
// once into shared memory, then runs the column pass and the row pass there.
//
// Reconstruction W = E^dagger S, per axis:
//     Ysyn(x) = sum_k a_lo[k] g_lo[x+2L'-2k-1] + a_hi[k] g_hi[x+2L'-2k-1]
//     out[t]  = (1/c[t]) * sum_{x : ext(x) = t} Ysyn(x),  x in [-L', N+L')
// (x is the extended coordinate shifted by L').  The fold E^dagger is a
// gather: a CTA computes Ysyn over its own rows plus, at the image border,
// the L' mirrored rows (symmetric case), so no atomics are needed.  The
// periodic extension's far copies and tiny images (N <= 2L') go through a
// per-pixel gather kernel.
#include <algorithm>
#include <type_traits>

#include "adjwt_internal.h"
#include "device_common.cuh"
#include "tma.cuh"

namespace adjwt {
namespace {

constexpr int kTile = kSynthTile;
constexpr int kThreads = 256;
constexpr int kAnaThreads = 288;  // analysis: 9 warps take the 4 x (2 kTile + L - 2) column items in one round

struct AnaArgs {
  const float* in;
  int in_pitch;
  int Nr, Nc, nr, nc, mode;
  const float* winv_r;
  const float* winv_c;
  float* dst[4];  // plain destinations (LL, LH, HL, HH)
  float* px[4];   // prox state buffers (non-null => prox band)
  float* py[4];
  int out_pitch;
  float step, thresh, beta;
  const double* beta_dev;  // non-null: beta from device memory
  double* l1;     // per-CTA partials (null = skip)
  float flo[kMaxTaps], fhi[kMaxTaps];
  int in_r0, in_r1, in_c0, in_c1, tiles_r, tiles_c;  // tiles left to the TMA kernel (see border_tile)
};


// Issue up to 8 independent gathers per thread before storing them, so the
// staging of a tile keeps several loads in flight.
// MAXN bounds `total` at compile time, so every load of a tile is issued
// before the first shared-memory store: one memory round trip per tile.
template <int MAXN, int NT = kThreads, typename Src, typename Dst>
__device__ __forceinline__ void staged_copy(int total, Src src, Dst dst) {
  constexpr int U = (MAXN + NT - 1) / NT;
  float v[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int i = threadIdx.x + u * NT;
    v[u] = i < total ? src(i) : 0.0f;
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int i = threadIdx.x + u * NT;
    if (i < total) dst(i, v[u]);
  }
}

// Tile of this CTA: blockIdx directly when no rectangle is left to a TMA
// kernel, else the i-th tile of the tiles_r x tiles_c grid outside the
// rectangle [r0, r1) x [c0, c1) (rows above, rows below, then the columns
// beside it).
__device__ __forceinline__ void border_tile(int r0, int r1, int c0, int c1, int tiles_r, int tiles_c, int* ty,
                                            int* tx) {
  if (r1 <= r0) {
    *ty = blockIdx.y;
    *tx = blockIdx.x;
    return;
  }
  const int i = blockIdx.x, TC = tiles_c;
  const int ntop = r0 * TC, nbot = (tiles_r - r1) * TC;
  if (i < ntop) {
    *ty = i / TC;
    *tx = i - *ty * TC;
  } else if (i < ntop + nbot) {
    const int j = i - ntop;
    *ty = r1 + j / TC;
    *tx = j - (*ty - r1) * TC;
  } else {
    const int j = i - ntop - nbot, side = c0 + (TC - c1);
    const int rr = j / side, k = j - rr * side;
    *ty = r0 + rr;
    *tx = k < c0 ? k : c1 + (k - c0);
  }
}

// ---------------------------------------------------------------- analysis
// One CTA: kTile x kTile outputs of each of the four bands.  Column pass:
// each thread filters kAP consecutive outputs of one column from 2*kAP + L - 2
// values held in registers; row pass likewise along a row (lanes on rows, odd
// row pitch).  Both filters of a pass share the loaded window.
constexpr int kAP = 8;
// prox epilogue: each row-pass thread's prox state (y and x of its two bands,
// 8 values each) is copied into its own dynamic-shared-memory slot at kernel
// start, so the loads overlap the window gather and both passes; 36-float
// slots put a quarter warp's 16-byte reads on distinct banks
constexpr int kProxSlot = 36;
constexpr int kProxRowers = 2 * (kTile / kAP) * 32;
constexpr size_t kProxSlotBytes = (size_t)kProxRowers * kProxSlot * sizeof(float);

// Loads of a level's input.  Inputs written before the launch take the
// read-only path; the level chain (below) reads LL bands that other CTAs of
// the same launch wrote, so it loads them at L2 (ld.global.cg), never from a
// possibly stale L1 or read-only cache line.
template <bool CG>
__device__ __forceinline__ float ld_level(const float* p) {
  if constexpr (CG) {
    return __ldcg(p);
  } else {
    return __ldg(p);
  }
}

// One kTile x kTile coefficient tile (tile_y, tile_x) of the four bands of
// one level; adds this thread's |x_k| to l1 when the prox runs.
template <int L, bool CG>
__device__ __forceinline__ void analysis_tile(const AnaArgs& a, int tile_y, int tile_x, float& l1) {
  constexpr int Lp = L - 1;
  constexpr int E = 2 * kTile + L - 2;  // extended samples feeding one tile
  constexpr int EP = E | 1;
  constexpr int NW = 2 * kAP + L - 2;   // window of one thread
  __shared__ float T[E][EP];
  __shared__ float V[2][kTile][EP];
  __shared__ int s_src[2][E];
  __shared__ float s_w[2][E];

  const int k0 = tile_y * kTile, l0 = tile_x * kTile;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  extern __shared__ float prox_slots[];  // kProxSlotBytes when the launch has prox bands, else none
  const bool rower = warp < 2 * (kTile / kAP);
  // row pass + prox epilogue: thread = (row kk, vertical filter f, block lb)
  const int kk = lane, f = warp & 1, lb = warp >> 1;
  const int k = k0 + kk, lbase = l0 + kAP * lb;
  const size_t row = (size_t)k * a.out_pitch + lbase;
  const bool full = lbase + kAP <= a.nc;   // all eight inside the band (16-byte aligned)
  const bool has_prox = a.px[1] != nullptr;
  // band pointers by compile-time index (avoids dynamic indexing of the parameter block)
  auto pick = [&](float* const (&arr)[4], int b) -> float* {
    return b == 0 ? arr[0] : (b == 1 ? arr[1] : (b == 2 ? arr[2] : arr[3]));
  };
  float* pxs[2] = {pick(a.px, f), pick(a.px, f + 2)};
  float* pys[2] = {pick(a.py, f), pick(a.py, f + 2)};
  float* slot = prox_slots + tid * kProxSlot;
  if (has_prox && rower && k < a.nr && lbase < a.out_pitch) {
#pragma unroll
    for (int hb = 0; hb < 2; ++hb) {
      if (!pxs[hb]) continue;
      if (full) {
#pragma unroll
        for (int q = 0; q < kAP / 4; ++q) {
          cp_async16(slot + hb * 16 + 4 * q, pys[hb] + row + 4 * q, 16u);
          cp_async16(slot + hb * 16 + 8 + 4 * q, pxs[hb] + row + 4 * q, 16u);
        }
      } else {
#pragma unroll
        for (int p = 0; p < kAP; ++p) {
          const bool in = lbase + p < a.nc;
          cp_async4(slot + hb * 16 + p, pys[hb] + row + (in ? p : 0), in ? 4u : 0u);
          cp_async4(slot + hb * 16 + 8 + p, pxs[hb] + row + (in ? p : 0), in ? 4u : 0u);
        }
      }
    }
    cp_async_commit();
  }

  // first extended coordinate of each axis and whether the tile reads only
  // plain interior samples (no zero, mirror, wrap or weight)
  const int e0r = 2 * k0 + 1 - Lp, e0c = 2 * l0 + 1 - Lp;
  const int sh = a.mode == 3 ? 0 : Lp;   // extended coordinate -> image index
  auto interior = [&](int e0, int N, const float* winv) {
    const int lo = e0 - sh, hi = e0 - sh + E - 1;
    const int guard = winv ? Lp : 0;
    return lo >= guard && hi < N - guard;
  };
  const bool fast = interior(e0r, a.Nr, a.winv_r) && interior(e0c, a.Nc, a.winv_c);

  if (fast) {
    const float* src = a.in + (size_t)(e0r - sh) * a.in_pitch + (e0c - sh);
    staged_copy<E * E, kAnaThreads>(
        E * E,
        [&](int i) {
          const int er = i / E;
          return ld_level<CG>(src + (size_t)er * a.in_pitch + (i - er * E));
        },
        [&](int i, float v) {
          const int er = i / E;
          T[er][i - er * E] = v;
        });
  } else {
    for (int i = tid; i < 2 * E; i += kAnaThreads) {
      const int axis = i / E, el = i - axis * E;
      const int e = (axis == 0 ? e0r : e0c) + el;
      const int N = axis == 0 ? a.Nr : a.Nc;
      int s;
      if (a.mode == 3) {
        s = pos_mod(e, N);
      } else {
        s = (e >= 0 && e < N + 2 * Lp) ? ext_src(e - Lp, N, a.mode) : -1;
      }
      const float* winv = axis == 0 ? a.winv_r : a.winv_c;
      s_src[axis][el] = s;
      s_w[axis][el] = (s >= 0 && winv) ? __ldg(winv + s) : 1.0f;
    }
    __syncthreads();
    staged_copy<E * E, kAnaThreads>(
        E * E,
        [&](int i) {
          const int er = i / E, ec = i - er * E;
          const int sr = s_src[0][er], sc = s_src[1][ec];
          return (sr >= 0 && sc >= 0) ? s_w[0][er] * s_w[1][ec] * ld_level<CG>(a.in + (size_t)sr * a.in_pitch + sc)
                                      : 0.0f;
        },
        [&](int i, float v) {
          const int er = i / E;
          T[er][i - er * E] = v;
        });
  }
  __syncthreads();

  // column pass: V[f][kk][ec] = sum_t f[t] T[2 kk + L' - t][ec]
  for (int item = tid; item < E * (kTile / kAP); item += kAnaThreads) {
    const int kb = item / E, ec = item - kb * E;
    float w[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) w[j] = T[2 * kAP * kb + j][ec];
#pragma unroll
    for (int p = 0; p < kAP; ++p) {
      float lo = 0.0f, hi = 0.0f;
#pragma unroll
      for (int t = 0; t < L; ++t) {
        lo = fmaf(a.flo[t], w[2 * p + Lp - t], lo);
        hi = fmaf(a.fhi[t], w[2 * p + Lp - t], hi);
      }
      V[0][kAP * kb + p][ec] = lo;
      V[1][kAP * kb + p][ec] = hi;
    }
  }
  __syncthreads();

  // row pass + store / prox epilogue: thread = (row kk, vertical filter f, block lb)
  // (l1: per-thread float32 partial of |x_k|, float64 across the block)
  const float beta = a.beta_dev ? static_cast<float>(*a.beta_dev) : a.beta;
  if (rower) {  // the ninth warp has no row-pass item
    float w[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) w[j] = V[f][kk][2 * kAP * lb + j];
    float res[2][kAP];
#pragma unroll
    for (int p = 0; p < kAP; ++p) {
      float lo = 0.0f, hi = 0.0f;
#pragma unroll
      for (int t = 0; t < L; ++t) {
        lo = fmaf(a.flo[t], w[2 * p + Lp - t], lo);
        hi = fmaf(a.fhi[t], w[2 * p + Lp - t], hi);
      }
      res[0][p] = lo;
      res[1][p] = hi;
    }
    if (k < a.nr && lbase < a.out_pitch) {
      float* dst[2] = {pick(a.dst, f), pick(a.dst, f + 2)};
      // prox bands: y and x from this thread's slot (copied at kernel start)
      float yv[2][kAP], xv[2][kAP];
      if (has_prox) cp_async_wait_all();
#pragma unroll
      for (int hb = 0; hb < 2; ++hb) {
        if (!pxs[hb]) continue;
#pragma unroll
        for (int q = 0; q < kAP / 4; ++q) {
          const float4 y4 = reinterpret_cast<const float4*>(slot + hb * 16)[q];
          const float4 x4 = reinterpret_cast<const float4*>(slot + hb * 16 + 8)[q];
          yv[hb][4 * q] = y4.x; yv[hb][4 * q + 1] = y4.y; yv[hb][4 * q + 2] = y4.z; yv[hb][4 * q + 3] = y4.w;
          xv[hb][4 * q] = x4.x; xv[hb][4 * q + 1] = x4.y; xv[hb][4 * q + 2] = x4.z; xv[hb][4 * q + 3] = x4.w;
        }
      }
#pragma unroll
      for (int hb = 0; hb < 2; ++hb) {
        if (pxs[hb]) {
          float* __restrict__ ys = pys[hb] + row;
          float* __restrict__ xs = pxs[hb] + row;
          float xn[kAP], yn[kAP];
#pragma unroll
          for (int p = 0; p < kAP; ++p) {
            const float v = yv[hb][p] - a.step * res[hb][p];
            const float mag = fabsf(v) - a.thresh;
            float x = mag > 0.0f ? copysignf(mag, v) : 0.0f;
            float y = fmaf(beta, x - xv[hb][p], x);
            if (!full && lbase + p >= a.nc) x = y = 0.0f;
            xn[p] = x;
            yn[p] = y;
            if (a.l1) l1 += fabsf(x);
          }
          if (full) {
#pragma unroll
            for (int q = 0; q < kAP / 4; ++q) {
              reinterpret_cast<float4*>(xs)[q] = make_float4(xn[4 * q], xn[4 * q + 1], xn[4 * q + 2], xn[4 * q + 3]);
              reinterpret_cast<float4*>(ys)[q] = make_float4(yn[4 * q], yn[4 * q + 1], yn[4 * q + 2], yn[4 * q + 3]);
            }
          } else {
#pragma unroll
            for (int p = 0; p < kAP; ++p) {
              if (lbase + p < a.out_pitch) {
                xs[p] = xn[p];
                ys[p] = yn[p];
              }
            }
          }
        } else if (dst[hb]) {
          float* d = dst[hb] + row;
          if (full) {
            reinterpret_cast<float4*>(d)[0] = make_float4(res[hb][0], res[hb][1], res[hb][2], res[hb][3]);
            reinterpret_cast<float4*>(d)[1] = make_float4(res[hb][4], res[hb][5], res[hb][6], res[hb][7]);
          } else {
#pragma unroll
            for (int p = 0; p < kAP; ++p)
              if (lbase + p < a.out_pitch) d[p] = lbase + p < a.nc ? res[hb][p] : 0.0f;
          }
        }
      }
    }
  }
}

template <int L>
__global__ void __launch_bounds__(kAnaThreads, 2) k_analysis(const AnaArgs a) {
  pdl_entry();
  __shared__ double red[kAnaThreads / 32];
  int tile_y, tile_x;
  border_tile(a.in_r0, a.in_r1, a.in_c0, a.in_c1, a.tiles_r, a.tiles_c, &tile_y, &tile_x);
  float l1 = 0.0f;
  analysis_tile<L, false>(a, tile_y, tile_x, l1);
  if (a.l1) {
    const double tot = block_sum<kAnaThreads>((double)l1, red);
    if (threadIdx.x == 0) a.l1[blockIdx.y * gridDim.x + blockIdx.x] = tot;
  }
}

struct SynArgs {
  const float* band[4];  // LL, LH, HL, HH of level j
  int band_pitch;
  float* out;
  int out_pitch;
  int Nr, Nc, nr, nc, mode;
  const float* winv_r;
  const float* winv_c;
  float g[2][kMaxTaps];  // synthesis filters lo / hi
  // tiles (kTile units) [in_r0, in_r1) x [in_c0, in_c1) are left to the TMA
  // kernel; the grid then enumerates the other tiles of the tiles_r x tiles_c
  // grid (rows above, rows below, then the columns beside the rectangle)
  int in_r0, in_r1, in_c0, in_c1, tiles_r, tiles_c;
};

// ---------------------------------------------------------------- synthesis
// One CTA: kTile x kTile output pixels.  Along an axis the outputs x of the
// tile's virtual range [xa, xb) come in pairs (xa + 2p, xa + 2p + 1); with
// phi = (xa + off - 1) mod 2 and Kb = floor((xa + off - 1) / 2) the pair p
// reads the coefficients Kb + p - q (+ e when phi = 1) with filter taps
// m = (e xor phi) + 2q, q < L/2.  A thread produces kSP pairs of one column
// (column pass) or one row (row pass) from kSP + L/2 coefficients per band
// held in registers.
constexpr int kSP = 4;

template <int L>
struct SynGeo {
  static constexpr int Lp = L - 1;
  static constexpr int XM = kTile + 2 * Lp;                   // virtual outputs per axis (max)
  static constexpr int NPAIR = (XM + 1) / 2;
  static constexpr int NBLK = (NPAIR + kSP - 1) / kSP;
  static constexpr int KM = NBLK * kSP + L / 2;               // coefficients per axis (max)
  static constexpr int KP = KM | 1;
  static constexpr int NC = kSP + L / 2;                      // coefficients per thread window
  static constexpr int YP = XM | 1;
};

template <int L, int PHI>
__device__ __forceinline__ void pair_block(const float (&c0)[SynGeo<L>::NC], const float (&c1)[SynGeo<L>::NC],
                                           const float (&g0)[L], const float (&g1)[L], float (&out)[2 * kSP]) {
#pragma unroll
  for (int p = 0; p < kSP; ++p) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      float acc = 0.0f;
#pragma unroll
      for (int q = 0; q < L / 2; ++q) {
        const int j = p - q + L / 2 - 1 + (PHI ? e : 0);
        const int m = (PHI ? 1 - e : e) + 2 * q;
        acc = fmaf(c0[j], g0[m], acc);
        acc = fmaf(c1[j], g1[m], acc);
      }
      out[2 * p + e] = acc;
    }
  }
}

// One kTile x kTile output tile (tile_y, tile_x) of one level.
template <int L, bool CG>
__device__ __forceinline__ void synthesis_tile(const SynArgs& a, int tile_y, int tile_x) {
  using G = SynGeo<L>;
  constexpr int Lp = L - 1;
  __shared__ float C[4][G::KM][G::KP];
  __shared__ float H[2][G::XM][G::KP];     // reused as Y[kTile][YP]
  __shared__ float Gf[2][kTile][G::KP];
  float(*Y)[G::YP] = reinterpret_cast<float(*)[G::YP]>(&H[0][0][0]);
  static_assert(kTile * G::YP <= 2 * G::XM * G::KP, "Y must fit in H");

  const int tid = threadIdx.x;
  const int t0r = tile_y * kTile, t0c = tile_x * kTile;
  const bool sym = a.mode == 1;
  float g0[L], g1[L];
#pragma unroll
  for (int t = 0; t < L; ++t) {
    g0[t] = a.g[0][t];
    g1[t] = a.g[1][t];
  }
  // filter index m = x + off - 2k - 1: the extended modes carry the L' shift of
  // the extension on top of the bank's delay L'; the circular mode has none
  const int off = a.mode == 3 ? Lp : 2 * Lp;
  int xa[2], nx[2], phi[2], ka[2], nk[2], nblk[2];
  {
    const int t0[2] = {t0r, t0c};
    const int N[2] = {a.Nr, a.Nc};
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
      xa[ax] = (sym && t0[ax] < Lp) ? -Lp : t0[ax];
      const int xb = (sym && t0[ax] + kTile > N[ax] - Lp) ? N[ax] + Lp : t0[ax] + kTile;
      nx[ax] = xb - xa[ax];
      phi[ax] = (xa[ax] + off - 1) & 1;
      const int Kb = floor_div(xa[ax] + off - 1, 2);
      nblk[ax] = ((nx[ax] + 1) / 2 + kSP - 1) / kSP;
      ka[ax] = Kb - (L / 2 - 1);
      nk[ax] = nblk[ax] * kSP + L / 2 - 1 + phi[ax];
    }
  }

  // Interior tiles (no mirror copy, weight 1, coefficients inside the bands,
  // no wrap) skip the fold buffers: the column pass writes the folded rows
  // directly and the row pass stores straight to global memory.
  bool fast = true;
  {
    const int t0[2] = {t0r, t0c};
    const int N[2] = {a.Nr, a.Nc};
    const int n[2] = {a.nr, a.nc};
    const bool weighted = a.winv_r != nullptr || a.mode == 2;
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
      const int guard = (weighted || sym) ? Lp : 0;
      fast = fast && xa[ax] == t0[ax] && nx[ax] == kTile && t0[ax] >= guard && t0[ax] + kTile <= N[ax] - guard &&
             ka[ax] >= 0 && ka[ax] + nk[ax] <= n[ax];
    }
  }
  if (fast) {
    // coefficients: warp w stages band w%4, rows of parity w/4; every load of
    // the thread is issued before its first shared-memory store
    constexpr int FK = 4 * kSP + L / 2;  // nk of an interior tile is at most this
    constexpr int RPW = (FK + 1) / 2;    // rows per warp
    const int lane = tid & 31, warp = tid >> 5;
    {
      const int b = warp & 3, half = warp >> 2;
      const float* src = a.band[b] + (size_t)(ka[0] + half) * a.band_pitch + ka[1] + lane;
      float v[RPW];
#pragma unroll
      for (int r = 0; r < RPW; ++r) {
        const int kk = half + 2 * r;
        v[r] = (kk < nk[0] && lane < nk[1]) ? ld_level<CG>(src + (size_t)(2 * r) * a.band_pitch) : 0.0f;
      }
#pragma unroll
      for (int r = 0; r < RPW; ++r) {
        const int kk = half + 2 * r;
        if (kk < nk[0] && lane < nk[1]) C[b][kk][lane] = v[r];
      }
    }
    __syncthreads();
    // column pass into the folded rows (identity fold, weight 1): warp = (hb, block), lane = column
    if (lane < nk[1]) {
      const int hb = warp & 1, blk = warp >> 1, ll = lane;
      float c0[G::NC], c1[G::NC], out[2 * kSP];
#pragma unroll
      for (int j = 0; j < G::NC; ++j) {
        const int kk = blk * kSP + j;
        c0[j] = kk < nk[0] ? C[2 * hb][kk][ll] : 0.0f;
        c1[j] = kk < nk[0] ? C[2 * hb + 1][kk][ll] : 0.0f;
      }
      if (phi[0])
        pair_block<L, 1>(c0, c1, g0, g1, out);
      else
        pair_block<L, 0>(c0, c1, g0, g1, out);
#pragma unroll
      for (int o = 0; o < 2 * kSP; ++o) Gf[hb][2 * kSP * blk + o][ll] = out[o];
    }
    __syncthreads();
    // row pass straight to global memory: eight consecutive pixels per thread
    for (int item = tid; item < kTile * nblk[1]; item += kThreads) {
      const int tt = item & (kTile - 1), blk = item / kTile;
      float c0[G::NC], c1[G::NC], out[2 * kSP];
#pragma unroll
      for (int j = 0; j < G::NC; ++j) {
        const int kk = blk * kSP + j;
        c0[j] = kk < nk[1] ? Gf[0][tt][kk] : 0.0f;
        c1[j] = kk < nk[1] ? Gf[1][tt][kk] : 0.0f;
      }
      if (phi[1])
        pair_block<L, 1>(c0, c1, g0, g1, out);
      else
        pair_block<L, 0>(c0, c1, g0, g1, out);
      float4* dst = reinterpret_cast<float4*>(a.out + (size_t)(t0r + tt) * a.out_pitch + t0c + 2 * kSP * blk);
      dst[0] = make_float4(out[0], out[1], out[2], out[3]);
      dst[1] = make_float4(out[4], out[5], out[6], out[7]);
    }
    return;
  }

  // weights 1/c of this tile's output rows and columns (fold E^dagger)
  __shared__ float s_wr[kTile], s_wc[kTile];
  if (tid < 2 * kTile) {
    const int ax = tid / kTile, u = tid - ax * kTile;
    const float* winv = ax ? a.winv_c : a.winv_r;
    const int t = (ax ? t0c : t0r) + u, N = ax ? a.Nc : a.Nr;
    (ax ? s_wc : s_wr)[u] = (winv && t < N) ? __ldg(winv + t) : 1.0f;
  }
  // coefficient tiles of the four bands (periodic wrap for PER, zeros
  // outside otherwise); compile-time strides keep the index arithmetic cheap
  constexpr int KK = G::KM * G::KM;
  staged_copy<4 * KK>(
      4 * KK,
      [&](int i) {
        const int b = i / KK, rem = i - b * KK;
        const int kk = rem / G::KM, ll = rem - kk * G::KM;
        if (kk >= nk[0] || ll >= nk[1]) return 0.0f;
        int k = ka[0] + kk, l = ka[1] + ll;
        if (a.mode == 3) {
          k = pos_mod(k, a.nr);
          l = pos_mod(l, a.nc);
        } else if (k < 0 || k >= a.nr || l < 0 || l >= a.nc) {
          return 0.0f;
        }
        return ld_level<CG>(a.band[b] + (size_t)k * a.band_pitch + l);
      },
      [&](int i, float v) {
        const int b = i / KK, rem = i - b * KK;
        const int kk = rem / G::KM;
        C[b][kk][rem - kk * G::KM] = v;
      });
  __syncthreads();

  // column pass: H[hb][x][l] over the virtual rows, both vertical bands summed
  for (int item = tid; item < 2 * G::KM * nblk[0]; item += kThreads) {
    const int blk = item / (2 * G::KM);
    const int rem = item - blk * 2 * G::KM;
    const int hb = rem / G::KM, ll = rem - hb * G::KM;
    if (ll >= nk[1]) continue;
    float c0[G::NC], c1[G::NC], out[2 * kSP];
#pragma unroll
    for (int j = 0; j < G::NC; ++j) {
      const int kk = blk * kSP + j;
      c0[j] = kk < nk[0] ? C[2 * hb][kk][ll] : 0.0f;
      c1[j] = kk < nk[0] ? C[2 * hb + 1][kk][ll] : 0.0f;
    }
    if (phi[0])
      pair_block<L, 1>(c0, c1, g0, g1, out);
    else
      pair_block<L, 0>(c0, c1, g0, g1, out);
#pragma unroll
    for (int o = 0; o < 2 * kSP; ++o) {
      const int xx = 2 * kSP * blk + o;
      if (xx < nx[0]) H[hb][xx][ll] = out[o];
    }
  }
  __syncthreads();

  // fold rows (E^dagger along the vertical axis)
  for (int i = tid; i < 2 * kTile * G::KM; i += kThreads) {
    const int hb = i / (kTile * G::KM);
    const int rem = i - hb * kTile * G::KM;
    const int tt = rem / G::KM, ll = rem - tt * G::KM;
    if (ll >= nk[1]) continue;
    const int t = t0r + tt;
    float v = 0.0f;
    if (t < a.Nr) {
      v = H[hb][t - xa[0]][ll];
      if (sym) {
        if (t < Lp) v += H[hb][-1 - t - xa[0]][ll];
        if (t >= a.Nr - Lp) v += H[hb][2 * a.Nr - 1 - t - xa[0]][ll];
      }
      v *= s_wr[tt];
    }
    Gf[hb][tt][ll] = v;
  }
  __syncthreads();

  // row pass: Y[t][x] over the virtual columns; lanes on rows
  for (int item = tid; item < kTile * nblk[1]; item += kThreads) {
    const int tt = item & (kTile - 1), blk = item / kTile;
    float c0[G::NC], c1[G::NC], out[2 * kSP];
#pragma unroll
    for (int j = 0; j < G::NC; ++j) {
      const int kk = blk * kSP + j;
      c0[j] = kk < nk[1] ? Gf[0][tt][kk] : 0.0f;
      c1[j] = kk < nk[1] ? Gf[1][tt][kk] : 0.0f;
    }
    if (phi[1])
      pair_block<L, 1>(c0, c1, g0, g1, out);
    else
      pair_block<L, 0>(c0, c1, g0, g1, out);
#pragma unroll
    for (int o = 0; o < 2 * kSP; ++o) {
      const int xx = 2 * kSP * blk + o;
      if (xx < nx[1]) Y[tt][xx] = out[o];
    }
  }
  __syncthreads();

  // fold columns and store (four consecutive pixels per thread)
  const bool ppd = a.mode == 2;
  for (int i = tid; i < kTile * (kTile / 4); i += kThreads) {
    const int tt = i / (kTile / 4), c4 = (i - tt * (kTile / 4)) * 4;
    const int tr = t0r + tt;
    if (tr >= a.Nr) continue;
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int tc = t0c + c4 + u;
      float s = 0.0f;
      if (tc < a.Nc) {
        s = Y[tt][tc - xa[1]];
        if (sym) {
          if (tc < Lp) s += Y[tt][-1 - tc - xa[1]];
          if (tc >= a.Nc - Lp) s += Y[tt][2 * a.Nc - 1 - tc - xa[1]];
        }
        s *= s_wc[c4 + u];
      }
      v[u] = s;
    }
    const bool ppd_row = ppd && (tr < Lp || tr >= a.Nr - Lp);
    float* dst = a.out + (size_t)tr * a.out_pitch + t0c + c4;
    if (!ppd && t0c + c4 + 4 <= a.Nc) {
      *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int tc = t0c + c4 + u;
        if (tc >= a.Nc) break;
        // pixels with periodic far copies belong to the border kernel
        if (ppd && (ppd_row || tc < Lp || tc >= a.Nc - Lp)) continue;
        dst[u] = v[u];
      }
    }
  }
}

template <int L>
__global__ void __launch_bounds__(kThreads) k_synthesis(const SynArgs a) {
  pdl_entry();
  int tile_y, tile_x;
  border_tile(a.in_r0, a.in_r1, a.in_c0, a.in_c1, a.tiles_r, a.tiles_c, &tile_y, &tile_x);
  synthesis_tile<L, false>(a, tile_y, tile_x);
}

// Per-pixel gather of W = E^dagger S for pixels with copies anywhere in the
// extended domain (periodic-extension borders, tiny images).
template <int L>
__global__ void __launch_bounds__(kThreads) k_synthesis_gather(const SynArgs a, int border_only, int64_t count) {
  pdl_entry();
  constexpr int Lp = L - 1;
  const int64_t idx = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (idx >= count) return;
  int tr, tc;
  if (!border_only) {
    tr = (int)(idx / a.Nc);
    tc = (int)(idx - (int64_t)tr * a.Nc);
  } else {
    const int64_t top = (int64_t)2 * Lp * a.Nc;
    if (idx < top) {
      const int row = (int)(idx / a.Nc);
      tr = row < Lp ? row : a.Nr - 2 * Lp + row;
      tc = (int)(idx - (int64_t)row * a.Nc);
    } else {
      const int64_t j = idx - top;
      tr = Lp + (int)(j / (2 * Lp));
      const int cc = (int)(j - (int64_t)(tr - Lp) * 2 * Lp);
      tc = cc < Lp ? cc : a.Nc - 2 * Lp + cc;
    }
  }
  // copies of t in [-L', N + L'): translation class (and mirror class for SYM)
  const int N[2] = {a.Nr, a.Nc};
  const int t[2] = {tr, tc};
  int xs[2][2 * kMaxTaps];
  int nx[2] = {0, 0};
#pragma unroll
  for (int ax = 0; ax < 2; ++ax) {
    const int P = a.mode == 1 ? 2 * N[ax] : (a.mode == 0 ? 0 : N[ax]);
    if (P == 0) {
      xs[ax][nx[ax]++] = t[ax];
      continue;
    }
    const int starts[2] = {t[ax], -1 - t[ax]};
    const int nclass = a.mode == 1 ? 2 : 1;
    for (int c = 0; c < nclass; ++c) {
      int x = starts[c] - P * floor_div(starts[c] + Lp, P);
      for (; x < N[ax] + Lp && nx[ax] < 2 * kMaxTaps; x += P) xs[ax][nx[ax]++] = x;
    }
  }
  float acc = 0.0f;
  for (int ir = 0; ir < nx[0]; ++ir) {
    const int xr = xs[0][ir];
    for (int ic = 0; ic < nx[1]; ++ic) {
      const int xc = xs[1][ic];
      for (int qr = 0; qr < L / 2; ++qr) {
        const int mr = ((xr + 1) & 1) + 2 * qr;
        const int k = (xr + 2 * Lp - 1 - mr) >> 1;
        if (k < 0 || k >= a.nr) continue;
        for (int qc = 0; qc < L / 2; ++qc) {
          const int mc = ((xc + 1) & 1) + 2 * qc;
          const int l = (xc + 2 * Lp - 1 - mc) >> 1;
          if (l < 0 || l >= a.nc) continue;
          const size_t o = (size_t)k * a.band_pitch + l;
#pragma unroll
          for (int va = 0; va < 2; ++va)
#pragma unroll
            for (int hb = 0; hb < 2; ++hb)
              acc = fmaf(__ldg(a.band[va + 2 * hb] + o), a.g[va][mr] * a.g[hb][mc], acc);
        }
      }
    }
  }
  if (a.winv_r) acc *= __ldg(a.winv_r + tr);
  if (a.winv_c) acc *= __ldg(a.winv_c + tc);
  a.out[(size_t)tr * a.out_pitch + tc] = acc;
}

// ---------------------------------------------------------------- level chain
// The deep levels of a transform move little data (LL_1 of a 2048^2 image is
// 4.3 MB and everything below it fits in L2), so one launch per level leaves
// them bound by launch latency and a dependent global round trip per level.
// The level chain runs a run of consecutive levels in one launch.  An item is
// one tile of one level; items are numbered level by level in the order the
// recursion needs them (W^*: j ascending, W: j descending).  A CTA takes the
// next item number from a counter, waits until every tile of the item's
// preceding level is done, runs the tile and counts it done.  A CTA only ever
// waits on items handed out before its own, to CTAs that are running, so the
// launch needs no co-residency and cannot deadlock with kernels of other
// streams.  Waits are bounded (kWaitCycles): a CTA that gives up records
// ADJWT_ERR_TIMEOUT in the device status word and stops taking items.
//
// Counters (ints, zeroed on the stream before each launch): [0] next item,
// [kChainDone + i] tiles of chain level i done.
constexpr int kChainDone = 4;

struct AnaChainArgs {
  AnaArgs lv[kMaxLevels];       // chain levels, shallowest first
  int first_item[kMaxLevels + 1];
  int nlev;
  int* counters;
  int* status;
  double* l1;                   // one float64 partial per CTA (null = none)
};

struct SynChainArgs {
  SynArgs lv[kMaxLevels];       // chain levels, deepest first
  int first_item[kMaxLevels + 1];
  int nlev;
  int* counters;
  int* status;
};

// Bounded wait (one thread) until *ctr >= target, with acquire semantics.
__device__ __forceinline__ bool chain_wait(const int* ctr, int target) {
  const long long t0 = clock64();
  for (;;) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
    if (v >= target) return true;
    if (clock64() - t0 > kWaitCycles) return false;
    __nanosleep(100);
  }
}

// Thread 0 takes the next item and waits for its level's inputs; every thread
// returns (item, level) or item = -1 when the chain is finished or a wait gave
// up.  The caller's next __syncthreads() must come after its last read of the
// shared words.
__device__ __forceinline__ void chain_next(const int* first_item, int nlev, int* counters, int* status, int* s_word,
                                           int* item_out, int* lev_out) {
  if (threadIdx.x == 0) {
    int item = atomicAdd(&counters[0], 1);
    int lev = 0;
    while (lev + 1 < nlev && item >= first_item[lev + 1]) ++lev;
    if (item >= first_item[nlev]) {
      item = -1;
    } else if (lev > 0 && !chain_wait(&counters[kChainDone + lev - 1], first_item[lev] - first_item[lev - 1])) {
      record_status(status, ADJWT_ERR_TIMEOUT);
      item = -1;
    }
    // (the acquire load of the wait, then the block barrier, orders every
    // thread's reads of the level's input after the producers' writes)
    s_word[0] = item;
    s_word[1] = lev;
  }
  __syncthreads();
  *item_out = s_word[0];
  *lev_out = s_word[1];
}

// Every write of the finished tile happens before the count is published
// (block barrier, then a device-scope fence by the counting thread).
__device__ __forceinline__ void chain_done(int* counters, int lev) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&counters[kChainDone + lev], 1);
  }
}

// Copy one level's argument block from the launch parameters into shared
// memory (the level index is only known at run time).
template <typename T, int NT>
__device__ __forceinline__ void copy_args(T* dst, const T* src) {
  static_assert(sizeof(T) % 4 == 0, "argument blocks are whole words");
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(T) / 4); i += NT) d[i] = s[i];
}

template <int L>
__global__ void __launch_bounds__(kAnaThreads, 2) k_analysis_chain(const __grid_constant__ AnaChainArgs c) {
  pdl_entry();
  __shared__ AnaArgs s_a;
  __shared__ int s_word[2];
  __shared__ double red[kAnaThreads / 32];
  double l1 = 0.0;  // float32 within a tile (as the per-level kernel), float64 across tiles
  int cur = -1;
  for (;;) {
    int item, lev;
    chain_next(c.first_item, c.nlev, c.counters, c.status, s_word, &item, &lev);
    if (item < 0) break;
    if (lev != cur) {
      copy_args<AnaArgs, kAnaThreads>(&s_a, &c.lv[lev]);
      __syncthreads();
      cur = lev;
    }
    const int local = item - c.first_item[lev];
    const int ty = local / s_a.tiles_c;
    float l1_tile = 0.0f;
    analysis_tile<L, true>(s_a, ty, local - ty * s_a.tiles_c, l1_tile);
    l1 += l1_tile;
    chain_done(c.counters, lev);
  }
  if (c.l1) {
    const double tot = block_sum<kAnaThreads>(l1, red);
    if (threadIdx.x == 0) c.l1[blockIdx.x] = tot;
  }
}

template <int L>
__global__ void __launch_bounds__(kThreads, 3) k_synthesis_chain(const __grid_constant__ SynChainArgs c) {
  pdl_entry();
  __shared__ SynArgs s_a;
  __shared__ int s_word[2];
  int cur = -1;
  for (;;) {
    int item, lev;
    chain_next(c.first_item, c.nlev, c.counters, c.status, s_word, &item, &lev);
    if (item < 0) break;
    if (lev != cur) {
      copy_args<SynArgs, kThreads>(&s_a, &c.lv[lev]);
      __syncthreads();
      cur = lev;
    }
    const int local = item - c.first_item[lev];
    const int ty = local / s_a.tiles_c;
    synthesis_tile<L, true>(s_a, ty, local - ty * s_a.tiles_c);
    chain_done(c.counters, lev);
  }
}

template <typename Fn>
int dispatch_L(int L, Fn&& fn) {
  switch (L) {
    case 2: return fn(std::integral_constant<int, 2>());
    case 4: return fn(std::integral_constant<int, 4>());
    case 8: return fn(std::integral_constant<int, 8>());
    case 10: return fn(std::integral_constant<int, 10>());
    default: return fail(ADJWT_ERR_INVALID_ARG, "unsupported filter length");
  }
}

int analysis_grid(const Level& L, dim3* g) {
  *g = dim3((L.band_pitch + kTile - 1) / kTile, (L.ax[0].n + kTile - 1) / kTile);
  return static_cast<int>(g->x * g->y);
}

// Arguments of the tiled reconstruction of level j (LL_j from the ping-pong
// buffer below level J, LL_{j-1} into the other buffer or the image).
SynArgs synth_args(const adjwt_wt_plan* p, int j, const float* coeffs, float* image, float* const llbuf[2]) {
  const Level& L = p->lv[j - 1];
  const FilterBank& fb = p->fb;
  SynArgs a{};
  for (int b = 0; b < 4; ++b) a.band[b] = (b == 0 && j < p->levels) ? llbuf[j % 2] : coeffs + L.off_band[b];
  a.band_pitch = L.band_pitch;
  a.out = (j == 1) ? image : llbuf[(j - 1) % 2];
  a.out_pitch = L.in_pitch;
  a.Nr = L.ax[0].N;
  a.Nc = L.ax[1].N;
  a.nr = L.ax[0].n;
  a.nc = L.ax[1].n;
  a.mode = p->bc;
  a.winv_r = L.ax[0].winv;
  a.winv_c = L.ax[1].winv;
  for (int t = 0; t < fb.L; ++t) {
    a.g[0][t] = static_cast<float>(fb.rec_lo[t]);
    a.g[1][t] = static_cast<float>(fb.rec_hi[t]);
  }
  return a;
}

template <typename K>
int resident_per_sm(K kernel, int threads, size_t dyn) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, dyn) != cudaSuccess) nb = 1;
  return std::max(1, nb);
}

// Counters of the level chain: the tail of the second LL buffer (reserved by
// the plan for transforms of two or more levels).
constexpr size_t kChainCounterBytes = (kChainDone + kMaxLevels) * sizeof(int);
int* chain_counters(const adjwt_wt_plan* p, float* llbuf1) {
  return reinterpret_cast<int*>(llbuf1 + p->ll_buf_floats[1] - kChainCounterFloats);
}

}  // namespace

// First level of the analysis-direction chain: the deepest run of levels
// (at least two) that no TMA kernel shares; levels + 1 when there is none.
int ana_chain_start(const adjwt_wt_plan* p, bool adjoint, bool prox) {
  if (p->chain_off) return p->levels + 1;
  int j0 = p->levels + 1;
  (void)adjoint;
  for (int j = p->levels; j >= 1; --j) {
    if (ana_tma_level(p, j, prox)) break;
    j0 = j;
  }
  return p->levels - j0 + 1 >= 2 ? j0 : p->levels + 1;
}

// The same for the reconstruction: levels without a TMA rectangle, the
// per-pixel gather path or the redundant-periodic border pass.
int syn_chain_start(const adjwt_wt_plan* p) {
  if (p->chain_off || p->bc == kPpd) return p->levels + 1;
  int j0 = p->levels + 1;
  for (int j = p->levels; j >= 1; --j) {
    int r0, r1, c0, c1;
    synth_tma_rect(p, j, &r0, &r1, &c0, &c1);
    if (r1 > r0 || p->lv[j - 1].generic_synth) break;
    j0 = j;
  }
  return p->levels - j0 + 1 >= 2 ? j0 : p->levels + 1;
}

// Per level: the tiled kernel's CTAs plus the TMA kernel's (at most one per
// 16 x 64 coefficient tile, which is no more than the 32 x 32 tile count).
int wt_l1_partial_slots(const adjwt_wt_plan* p) {
  int total = 0;
  for (const Level& L : p->lv) {
    dim3 g;
    total += 2 * analysis_grid(L, &g);
  }
  return total;
}

int launch_wt_analysis(const adjwt_wt_plan* p, const float* image, float* coeffs, bool adjoint,
                       const ProxArgs& prox, float* llbuf0, float* llbuf1, cudaStream_t s, int* l1_slots_used) {
  float* llbuf[2] = {llbuf0, llbuf1};
  const FilterBank& fb = p->fb;
  int slot = 0;
  const int j0 = ana_chain_start(p, adjoint, prox.x != nullptr);
  AnaChainArgs chain{};
  for (int j = 1; j <= p->levels; ++j) {
    const Level& L = p->lv[j - 1];
    AnaArgs a{};
    a.in = (j == 1) ? image : llbuf[(j - 1) % 2];
    a.in_pitch = L.in_pitch;
    a.Nr = L.ax[0].N;
    a.Nc = L.ax[1].N;
    a.nr = L.ax[0].n;
    a.nc = L.ax[1].n;
    a.mode = p->bc;
    a.winv_r = adjoint ? L.ax[0].winv : nullptr;
    a.winv_c = adjoint ? L.ax[1].winv : nullptr;
    a.out_pitch = L.band_pitch;
    for (int b = 0; b < 4; ++b) {
      const bool final_band = (b > 0) || (j == p->levels);
      float* base = nullptr;
      if (final_band) {
        if (prox.x) {
          a.px[b] = prox.x + L.off_band[b];
          a.py[b] = prox.y + L.off_band[b];
        } else {
          base = coeffs + L.off_band[b];
        }
      } else {
        base = llbuf[j % 2];
      }
      a.dst[b] = base;
    }
    a.step = prox.step;
    a.thresh = prox.thresh;
    a.beta = prox.beta;
    a.beta_dev = prox.beta_dev;
    for (int t = 0; t < fb.L; ++t) {
      if (adjoint) {  // dual analysis filters: synthesis filters reversed (Eq. 3, Eq. 4)
        a.flo[t] = static_cast<float>(fb.rec_lo[fb.L - 1 - t]);
        a.fhi[t] = static_cast<float>(fb.rec_hi[fb.L - 1 - t]);
      } else {
        a.flo[t] = static_cast<float>(fb.dec_lo[t]);
        a.fhi[t] = static_cast<float>(fb.dec_hi[t]);
      }
    }
    dim3 grid;
    int ncta = analysis_grid(L, &grid);
    a.tiles_c = grid.x;
    a.tiles_r = grid.y;
    if (j >= j0) {  // a level of the chain: its tiles become items of one launch
      const int i = j - j0;
      chain.lv[i] = a;
      // the tile code only tests l1 for null; the chain writes one partial per CTA
      chain.lv[i].l1 = (prox.x && prox.l1_partials) ? prox.l1_partials : nullptr;
      chain.first_item[i + 1] = chain.first_item[i] + ncta;
      continue;
    }
    const bool tma = ana_tma_level(p, j, prox.x != nullptr);  // the whole level on the TMA kernel
    if (tma) ncta = 0;
    const bool want_l1 = prox.x && prox.l1_partials;
    a.l1 = want_l1 ? prox.l1_partials + slot : nullptr;
    slot += ncta;
    const char* name = !adjoint ? "wt_analysis" : (prox.x ? "wt_adjoint_prox" : "wt_adjoint");
    if (ncta > 0) {
      int rc = dispatch_L(fb.L, [&](auto Lc) -> int {
        auto kern = k_analysis<decltype(Lc)::value>;
        const size_t dyn = prox.x ? kProxSlotBytes : 0;
        if (dyn) ADJWT_CUDA_CHECK(set_smem(kern, dyn));
        ADJWT_TRACED(name, j, s, pdl_launch(kern, grid, kAnaThreads, dyn, s, a));
        return ADJWT_OK;
      });
      if (rc) return rc;
      ADJWT_CUDA_CHECK(cudaGetLastError());
    }
    if (tma) {
      int used = 0;
      const char* tname = !adjoint ? "wt_analysis_tma" : (prox.x ? "wt_adjoint_prox_tma" : "wt_adjoint_tma");
      int rc = launch_ana_tma(p, j, adjoint, a.in, a.in_pitch, a.dst, a.px, a.py, a.out_pitch, a.step, a.thresh,
                              a.beta, a.beta_dev, want_l1 ? prox.l1_partials + slot : nullptr, a.flo, a.fhi, tname,
                              s, &used);
      if (rc) return rc;
      slot += used;
    }
  }
  if (j0 <= p->levels) {
    chain.nlev = p->levels - j0 + 1;
    chain.counters = chain_counters(p, llbuf1);
    chain.status = device_status_ptr();
    const char* name = !adjoint ? "wt_analysis_chain" : (prox.x ? "wt_adjoint_prox_chain" : "wt_adjoint_chain");
    const char* rname =
        !adjoint ? "wt_analysis_chain_reset" : (prox.x ? "wt_adjoint_prox_chain_reset" : "wt_adjoint_chain_reset");
    cudaError_t me = cudaSuccess;
    ADJWT_TRACED(rname, j0, s, me = cudaMemsetAsync(chain.counters, 0, kChainCounterBytes, s));
    ADJWT_CUDA_CHECK(me);
    int rc = dispatch_L(fb.L, [&](auto Lc) -> int {
      auto kern = k_analysis_chain<decltype(Lc)::value>;
      const size_t dyn = prox.x ? kProxSlotBytes : 0;
      if (dyn) ADJWT_CUDA_CHECK(set_smem(kern, dyn));
      const int per_sm = resident_per_sm(kern, kAnaThreads, dyn);  // after the attribute: it bounds the query
      const int ncta = std::max(1, std::min(chain.first_item[chain.nlev], per_sm * sm_count()));
      chain.l1 = (prox.x && prox.l1_partials) ? prox.l1_partials + slot : nullptr;
      slot += ncta;
      ADJWT_TRACED(name, j0, s, pdl_launch(kern, dim3(ncta), kAnaThreads, dyn, s, chain));
      return ADJWT_OK;
    });
    if (rc) return rc;
    ADJWT_CUDA_CHECK(cudaGetLastError());
  }
  if (l1_slots_used) *l1_slots_used = slot;
  return ADJWT_OK;
}

int launch_wt_synth(const adjwt_wt_plan* p, const float* coeffs, float* image, float* llbuf0, float* llbuf1,
                    cudaStream_t s) {
  float* llbuf[2] = {llbuf0, llbuf1};
  const FilterBank& fb = p->fb;
  const int Lp = fb.L - 1;
  const int j0 = syn_chain_start(p);
  if (j0 <= p->levels) {  // levels J .. j0 in one launch
    SynChainArgs chain{};
    chain.nlev = p->levels - j0 + 1;
    for (int j = p->levels; j >= j0; --j) {
      const int i = p->levels - j;
      chain.lv[i] = synth_args(p, j, coeffs, image, llbuf);
      SynArgs& a = chain.lv[i];
      a.tiles_c = (a.Nc + kTile - 1) / kTile;
      a.tiles_r = (a.Nr + kTile - 1) / kTile;
      chain.first_item[i + 1] = chain.first_item[i] + a.tiles_c * a.tiles_r;
    }
    chain.counters = chain_counters(p, llbuf1);
    chain.status = device_status_ptr();
    cudaError_t me = cudaSuccess;
    ADJWT_TRACED("wt_synth_chain_reset", j0, s, me = cudaMemsetAsync(chain.counters, 0, kChainCounterBytes, s));
    ADJWT_CUDA_CHECK(me);
    int rc = dispatch_L(fb.L, [&](auto Lc) -> int {
      auto kern = k_synthesis_chain<decltype(Lc)::value>;
      const int per_sm = resident_per_sm(kern, kThreads, 0);
      const int ncta = std::max(1, std::min(chain.first_item[chain.nlev], per_sm * sm_count()));
      ADJWT_TRACED("wt_synth_chain", j0, s, pdl_launch(kern, dim3(ncta), kThreads, 0, s, chain));
      return ADJWT_OK;
    });
    if (rc) return rc;
    ADJWT_CUDA_CHECK(cudaGetLastError());
  }
  for (int j = std::min(p->levels, j0 - 1); j >= 1; --j) {
    const Level& L = p->lv[j - 1];
    SynArgs a = synth_args(p, j, coeffs, image, llbuf);
    int rc = dispatch_L(fb.L, [&](auto Lc) -> int {
      constexpr int LL = decltype(Lc)::value;
      if (L.generic_synth) {
        const int64_t count = (int64_t)a.Nr * a.Nc;
        const unsigned nb = (unsigned)((count + kThreads - 1) / kThreads);
        ADJWT_TRACED("wt_synth_gather", j, s, pdl_launch(k_synthesis_gather<LL>, nb, kThreads, 0, s, a, 0, count));
      } else {
        a.tiles_c = (a.Nc + kTile - 1) / kTile;
        a.tiles_r = (a.Nr + kTile - 1) / kTile;
        int r0, r1, c0, c1;
        synth_tma_rect(p, j, &r0, &r1, &c0, &c1);
        dim3 grid(a.tiles_c, a.tiles_r);
        if (r1 > r0) {
          a.in_r0 = r0 / kTile;
          a.in_r1 = r1 / kTile;
          a.in_c0 = c0 / kTile;
          a.in_c1 = c1 / kTile;
          grid = dim3(a.tiles_r * a.tiles_c - (a.in_r1 - a.in_r0) * (a.in_c1 - a.in_c0), 1);
        }
        if (grid.x > 0)
          ADJWT_TRACED("wt_synth", j, s, pdl_launch(k_synthesis<LL>, grid, kThreads, 0, s, a));
        if (r1 > r0) {
          ADJWT_CUDA_CHECK(cudaGetLastError());
          int rc = launch_synth_tma(p, j, a.band, a.out, a.out_pitch, s);
          if (rc) return rc;
        }
        if (p->bc == kPpd) {
          const int64_t count = (int64_t)2 * Lp * a.Nc + (int64_t)(a.Nr - 2 * Lp) * 2 * Lp;
          const unsigned nb = (unsigned)((count + kThreads - 1) / kThreads);
          ADJWT_TRACED("wt_synth_gather", j, s, pdl_launch(k_synthesis_gather<LL>, nb, kThreads, 0, s, a, 1, count));
        }
      }
      return ADJWT_OK;
    });
    if (rc) return rc;
    ADJWT_CUDA_CHECK(cudaGetLastError());
  }
  return ADJWT_OK;
}

}  // namespace adjwt
