// Tiled bodies of one wavelet level (Sec. I-A, Eq. 2-4): the analysis
// direction W^* / W^dagger (with the FISTA prox epilogue on final bands) and
// the reconstruction W = E^dagger S, one kTile x kTile tile per call.  Each
// body is written for a block of NT threads (256, or 288 for the per-level
// analysis kernel) and works in shared memory the caller provides, so that
// the per-level kernels (wt_kernels.cu), the level chain and the batched
// FISTA engine (fista_batch.cu) run the same code.
//
// Analysis direction, one level, per axis:
//     out[k] = sum_i f[i] z[2k+1-i],   z[e] = w(e) * y[src(e)]
// with e the coordinate of the length N + 2L' extended signal, src(e) the
// extension map (zero / half-point symmetric / periodic) and w = 1/c for W^*
// (the weighted extension (E^dagger)^*, Eq. 2) or 1 for W^dagger; f are the
// dual analysis filters (reversed synthesis filters, Eq. 3 / Eq. 4) for W^*
// and the analysis filters for W^dagger.  The extension is applied in the
// load path.
//
// Reconstruction W = E^dagger S, per axis:
//     Ysyn(x) = sum_k a_lo[k] g_lo[x+2L'-2k-1] + a_hi[k] g_hi[x+2L'-2k-1]
//     out[t]  = (1/c[t]) * sum_{x : ext(x) = t} Ysyn(x),  x in [-L', N+L')
// The fold E^dagger is a gather: a tile computes Ysyn over its own rows plus,
// at the image border, the L' mirrored rows (symmetric case).
#pragma once

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
  int* status;  // device status word (checked builds record ADJWT_ERR_BOUNDS here)
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
// start, so the loads overlap the window gather and both passes.  A slot is
// eight 16-byte chunks; chunk c of thread t sits at position c xor (t mod 8),
// which puts a quarter warp's 16-byte reads of one chunk on distinct banks.
constexpr int kProxSlot = 32;
__device__ __forceinline__ float* prox_chunk(float* slot, int c) { return slot + 4 * (c ^ (threadIdx.x & 7)); }
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

// Shared memory of one analysis tile (the caller's: static in the per-level
// kernel, part of a dynamic buffer elsewhere).
template <int L>
struct AnaSmem {
  static constexpr int E = 2 * kTile + L - 2;  // extended samples feeding one tile
  static constexpr int EP = E | 1;
  float T[E][EP];
  float V[2][kTile][EP];
  int s_src[2][E];
  float s_w[2][E];
};

// One kTile x kTile coefficient tile (tile_y, tile_x) of the four bands of
// one level; adds this thread's |x_k| to l1 when the prox runs.  prox_slots:
// kProxSlotBytes of shared memory when the level has prox bands.
template <int L, bool CG, int NT = kAnaThreads>
__device__ __forceinline__ void analysis_tile(const AnaArgs& a, int tile_y, int tile_x, float& l1, AnaSmem<L>& sm,
                                              float* prox_slots) {
  constexpr int Lp = L - 1;
  constexpr int E = AnaSmem<L>::E;
  constexpr int NW = 2 * kAP + L - 2;   // window of one thread
  auto& T = sm.T;
  auto& V = sm.V;
  auto& s_src = sm.s_src;
  auto& s_w = sm.s_w;

  const int k0 = tile_y * kTile, l0 = tile_x * kTile;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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
  if (has_prox && rower && k < a.nr && lbase < a.out_pitch &&
      in_bounds(a.status, !full || lbase + kAP <= a.out_pitch)) {
#pragma unroll
    for (int hb = 0; hb < 2; ++hb) {
      if (!pxs[hb]) continue;
      if (full) {
#pragma unroll
        for (int q = 0; q < kAP / 4; ++q) {
          cp_async16(prox_chunk(slot, hb * 4 + q), pys[hb] + row + 4 * q, 16u);
          cp_async16(prox_chunk(slot, hb * 4 + 2 + q), pxs[hb] + row + 4 * q, 16u);
        }
      } else if constexpr (CG) {
        // state written earlier in the same launch: read at L2, never through L1
#pragma unroll
        for (int p = 0; p < kAP; ++p) {
          const bool in = lbase + p < a.nc;
          prox_chunk(slot, hb * 4 + p / 4)[p % 4] = in ? __ldcg(pys[hb] + row + p) : 0.0f;
          prox_chunk(slot, hb * 4 + 2 + p / 4)[p % 4] = in ? __ldcg(pxs[hb] + row + p) : 0.0f;
        }
      } else {
#pragma unroll
        for (int p = 0; p < kAP; ++p) {
          const bool in = lbase + p < a.nc;
          cp_async4(prox_chunk(slot, hb * 4 + p / 4) + p % 4, pys[hb] + row + (in ? p : 0), in ? 4u : 0u);
          cp_async4(prox_chunk(slot, hb * 4 + 2 + p / 4) + p % 4, pxs[hb] + row + (in ? p : 0), in ? 4u : 0u);
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
    staged_copy<E * E, NT>(
        E * E,
        [&](int i) {
          const int er = i / E, ec = i - er * E;
          const int ir = e0r - sh + er, ic = e0c - sh + ec;  // image row / column (the tile is interior)
          return in_bounds(a.status, ir >= 0 && ir < a.Nr && ic >= 0 && ic < a.Nc)
                     ? ld_level<CG>(src + (size_t)er * a.in_pitch + ec)
                     : 0.0f;
        },
        [&](int i, float v) {
          const int er = i / E;
          T[er][i - er * E] = v;
        });
  } else {
    for (int i = tid; i < 2 * E; i += NT) {
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
    staged_copy<E * E, NT>(
        E * E,
        [&](int i) {
          const int er = i / E, ec = i - er * E;
          const int sr = s_src[0][er], sc = s_src[1][ec];
          return (sr >= 0 && sc >= 0 && in_bounds(a.status, sr < a.Nr && sc < a.Nc))
                     ? s_w[0][er] * s_w[1][ec] * ld_level<CG>(a.in + (size_t)sr * a.in_pitch + sc)
                     : 0.0f;
        },
        [&](int i, float v) {
          const int er = i / E;
          T[er][i - er * E] = v;
        });
  }
  __syncthreads();

  // column pass: V[f][kk][ec] = sum_t f[t] T[2 kk + L' - t][ec]
  for (int item = tid; item < E * (kTile / kAP); item += NT) {
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
  float beta = a.beta;
  if (a.beta_dev) beta = static_cast<float>(CG ? __ldcg(a.beta_dev) : *a.beta_dev);
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
    if (k < a.nr && lbase < a.out_pitch && in_bounds(a.status, !full || lbase + kAP <= a.out_pitch)) {
      float* dst[2] = {pick(a.dst, f), pick(a.dst, f + 2)};
      // prox bands: y and x from this thread's slot (copied at kernel start)
      float yv[2][kAP], xv[2][kAP];
      if (has_prox) cp_async_wait_all();
#pragma unroll
      for (int hb = 0; hb < 2; ++hb) {
        if (!pxs[hb]) continue;
#pragma unroll
        for (int q = 0; q < kAP / 4; ++q) {
          const float4 y4 = *reinterpret_cast<const float4*>(prox_chunk(slot, hb * 4 + q));
          const float4 x4 = *reinterpret_cast<const float4*>(prox_chunk(slot, hb * 4 + 2 + q));
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
  int* status;  // device status word (checked builds record ADJWT_ERR_BOUNDS here)
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

// Shared memory of one reconstruction tile (the caller's).
template <int L>
struct SynSmem {
  using G = SynGeo<L>;
  float C[4][G::KM][G::KP];
  float H[2][G::XM][G::KP];     // reused as Y[kTile][YP]
  float Gf[2][kTile][G::KP];
  float s_wr[kTile], s_wc[kTile];
};

// One kTile x kTile output tile (tile_y, tile_x) of one level.
template <int L, bool CG>
__device__ __forceinline__ void synthesis_tile(const SynArgs& a, int tile_y, int tile_x, SynSmem<L>& sm) {
  using G = SynGeo<L>;
  constexpr int Lp = L - 1;
  auto& C = sm.C;
  auto& H = sm.H;
  auto& Gf = sm.Gf;
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
        const bool take = kk < nk[0] && lane < nk[1] &&
                          in_bounds(a.status, ka[0] + kk < a.nr && ka[1] + lane < a.nc && ka[0] >= 0 && ka[1] >= 0);
        v[r] = take ? ld_level<CG>(src + (size_t)(2 * r) * a.band_pitch) : 0.0f;
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
      if (!in_bounds(a.status, t0r + tt < a.Nr && t0c + 2 * kSP * (blk + 1) <= a.out_pitch)) continue;
      float4* dst = reinterpret_cast<float4*>(a.out + (size_t)(t0r + tt) * a.out_pitch + t0c + 2 * kSP * blk);
      dst[0] = make_float4(out[0], out[1], out[2], out[3]);
      dst[1] = make_float4(out[4], out[5], out[6], out[7]);
    }
    return;
  }

  // weights 1/c of this tile's output rows and columns (fold E^dagger)
  auto& s_wr = sm.s_wr;
  auto& s_wc = sm.s_wc;
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
        if (!in_bounds(a.status, k >= 0 && k < a.nr && l >= 0 && l < a.nc)) return 0.0f;
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
          if (tc < Lp && in_bounds(a.status, -1 - tc - xa[1] >= 0 && -1 - tc - xa[1] < nx[1]))
            s += Y[tt][-1 - tc - xa[1]];
          if (tc >= a.Nc - Lp && in_bounds(a.status, 2 * a.Nc - 1 - tc - xa[1] < nx[1]))
            s += Y[tt][2 * a.Nc - 1 - tc - xa[1]];
        }
        s *= s_wc[c4 + u];
      }
      v[u] = s;
    }
    const bool ppd_row = ppd && (tr < Lp || tr >= a.Nr - Lp);
    float* dst = a.out + (size_t)tr * a.out_pitch + t0c + c4;
    if (!ppd && t0c + c4 + 4 <= a.Nc) {
      if (in_bounds(a.status, t0c + c4 + 4 <= a.out_pitch))
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


// W = E^dagger S at one output pixel (tr, tc) by gathering every copy of it in
// the extended domain (periodic-extension borders, tiny images, symmetric
// levels whose mirror copies straddle a tile boundary).
template <int L, bool CG>
__device__ __forceinline__ void synthesis_gather_pixel(const SynArgs& a, int tr, int tc) {
  constexpr int Lp = L - 1;
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
              acc = fmaf(ld_level<CG>(a.band[va + 2 * hb] + o), a.g[va][mr] * a.g[hb][mc], acc);
        }
      }
    }
  }
  if (a.winv_r) acc *= __ldg(a.winv_r + tr);
  if (a.winv_c) acc *= __ldg(a.winv_c + tc);
  if (in_bounds(a.status, tr >= 0 && tr < a.Nr && tc >= 0 && tc < a.Nc)) a.out[(size_t)tr * a.out_pitch + tc] = acc;
}

}  // namespace
}  // namespace adjwt
