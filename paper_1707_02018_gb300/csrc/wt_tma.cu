// Persistent TMA-staged reconstruction W = E^dagger S for the full tiles of a
// level that need no fold and no weight: every full tile under the zero and
// circular extensions (band cells outside the band are zero, or wrapped by
// the threads after the copy), the interior tiles under the symmetric and
// redundant periodic ones.  The tiled kernel of wt_kernels.cu takes the
// remaining tiles of the level.
//
// Output tiles are kTH x kTW pixels of LL_{j-1}.  Along an axis, the outputs
// of a tile starting at an even t0 come in pairs (t0 + 2p, t0 + 2p + 1) that
// read the coefficients Kb + p - q (+ e when phi = 1), q < L/2, with filter
// taps (e xor phi) + 2q, Kb = floor((t0 + off - 1)/2) (off = 2L' for the
// extended modes, L' for PER); phi is the same for every tile of a level.
// The four band tiles a tile needs (rows ka_r .. ka_r + BR, columns from ka_c
// rounded down to 16 bytes) are copied by the TMA unit into one of two
// staging buffers while the CTA reconstructs the previous tile:
//   column pass: per horizontal band pair (LL,LH) / (HL,HH), a thread makes
//                16 consecutive rows of one coefficient column from a
//                register window (lanes on consecutive columns);
//   row pass:    a thread makes 16 consecutive pixels of one row (lanes on
//                rows, odd pitch) into the output tile, staged as four
//                32 x 32 boxes under the 128-byte swizzle in the staging
//                buffer the column pass has consumed; one thread then writes
//                them with TMA stores, and the next tile's copy goes into the
//                other buffer once the stores of the tile before have read it.
#include <algorithm>
#include <cstring>

#include "adjwt_internal.h"
#include "device_common.cuh"
#include "tma.cuh"

namespace adjwt {
namespace {

constexpr int kTH = 32;    // output rows per tile
constexpr int kTW = 128;   // output columns per tile
constexpr int kP = 8;      // output pairs per thread and pass
constexpr int kNT = 288;   // 9 warps: column-pass items; 8 of them in the row pass
constexpr int kSplitMin = 1536;  // W: levels shared with the tiled kernel; W^*: levels on the TMA kernel
constexpr int kWrapCols = 16;  // PER: the box of a full tile overhangs the band end by at most
constexpr int kWrapRows = 8;   // this many columns / rows (checked on the host)

__host__ __device__ constexpr int up4(int v) { return (v + 3) / 4 * 4; }
__host__ __device__ constexpr int up32(int v) { return (v + 31) / 32 * 32; }

template <int L>
struct SG {
  static constexpr int NC = kP + L / 2;             // coefficient window per thread
  static constexpr int BR = kTH / 2 + L / 2 + 1;    // staged band rows (>= every window row)
  static constexpr int BC = up4(3 + kTW / 2 + L / 2 + 1);  // staged band columns (16-byte start slack)
  static constexpr int BOX = BR * BC;                // floats of one band box
  static constexpr int BAND = up32(BOX);             // band stride in a buffer (128-byte aligned)
  static constexpr int BUF = 4 * BAND;               // floats per staging buffer (4 bands)
  static constexpr int NKC = kTW / 2 + L / 2;       // coefficient columns of the column pass (max)
  static constexpr int GP = (NKC + 1) | 1;          // odd pitch of the column-pass output
  // the output tile is staged as four 32 x 32 boxes (128-byte rows, 128-byte
  // swizzle) in the staging buffer the column pass has consumed, from a
  // 1024-byte boundary inside it
  static constexpr int OUT0 = 0;
  static constexpr int OUT1 = (BUF + 255) / 256 * 256;
  static_assert(kTH * kTW <= BUF && OUT1 + kTH * kTW <= 2 * BUF, "the staged output tile fits");
  static constexpr size_t smem_bytes() { return 1024 + (size_t)(2 * BUF + 2 * kTH * GP) * 4; }
};

struct SynTmaArgs {
  float* out;
  int out_pitch;
  int phi_r, phi_c;       // pair phase per axis
  int ka_r0, ka_c0;       // first coefficient of tile 0 minus t0/2, per axis
  int d_c;                // ka_c minus its 16-byte-aligned start
  int nk_c;               // coefficient columns used by a tile
  int ty0, tx0, ntx, ntiles;  // tile rectangle (tile units)
  int wrap;               // PER: overhanging band cells wrap around
  int nr, nc, band_pitch; // band extents (for the wrap fill)
  const float* band[4];
  int* status;
  float g[2][kMaxTaps];   // synthesis filters lo / hi
};

// 2 kP outputs from two coefficient windows (pairs p: outputs 2p, 2p+1)
template <int L, int PHI>
__device__ __forceinline__ void pairs(const float (&c0)[SG<L>::NC], const float (&c1)[SG<L>::NC],
                                      const SynTmaArgs& a, float (&out)[2 * kP]) {
#pragma unroll
  for (int p = 0; p < kP; ++p) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      float acc = 0.0f;
#pragma unroll
      for (int q = 0; q < L / 2; ++q) {
        const int j = p - q + L / 2 - 1 + (PHI ? e : 0);
        const int m = (PHI ? 1 - e : e) + 2 * q;
        acc = fmaf(c0[j], a.g[0][m], acc);
        acc = fmaf(c1[j], a.g[1][m], acc);
      }
      out[2 * p + e] = acc;
    }
  }
}

template <int L>
__global__ void __launch_bounds__(kNT, 3) k_synth_tma(const __grid_constant__ CUtensorMap m0,
                                                      const __grid_constant__ CUtensorMap m1,
                                                      const __grid_constant__ CUtensorMap m2,
                                                      const __grid_constant__ CUtensorMap m3,
                                                      const __grid_constant__ CUtensorMap mo, const SynTmaArgs a) {
  pdl_entry();
  using G = SG<L>;
  extern __shared__ unsigned char dyn[];
  __shared__ uint64_t bar[2];
  float* buf0 = reinterpret_cast<float*>(dyn + ((1024 - (smem_u32(dyn) & 1023)) & 1023));
  float* Gf = buf0 + 2 * G::BUF;  // [2][kTH][GP]
  const int tid = threadIdx.x;

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();

  uint32_t phase = 0, pending = 0;
  auto tile_origin = [&](int t, int& t0r, int& t0c) {
    const int ty = t / a.ntx;
    t0r = (a.ty0 + ty) * kTH;
    t0c = (a.tx0 + t - ty * a.ntx) * kTW;
  };
  auto issue = [&](int t, int b) {
    int t0r, t0c;
    tile_origin(t, t0r, t0c);
    if (tid == 0) {
      const int y = t0r / 2 + a.ka_r0, x = t0c / 2 + a.ka_c0 - a.d_c;
      float* dst = buf0 + b * G::BUF;
      fence_proxy_async();
      mbar_arrive_expect_tx(&bar[b], 4 * G::BOX * 4);
      tma_load_2d(dst, &m0, &bar[b], x, y);
      tma_load_2d(dst + G::BAND, &m1, &bar[b], x, y);
      tma_load_2d(dst + 2 * G::BAND, &m2, &bar[b], x, y);
      tma_load_2d(dst + 3 * G::BAND, &m3, &bar[b], x, y);
    }
    pending |= 1u << b;
  };

  int t = blockIdx.x, b = 0;
  if (t < a.ntiles) issue(t, 0);
  for (; t < a.ntiles; t += gridDim.x, b ^= 1) {
    int t0r, t0c;
    tile_origin(t, t0r, t0c);
    // PER: band cells of the box past the band end (zero-filled by the copy)
    // take their circularly wrapped values.  For full tiles the overhang is at
    // most kWrapCols columns and kWrapRows rows (one wrap); the cells are
    // fetched into registers while the copy is in flight.
    constexpr int RS = G::BR * kWrapCols, BS = kWrapRows * G::BC;
    constexpr int NRS = (4 * RS + kNT - 1) / kNT, NBS = (4 * BS + kNT - 1) / kNT;
    const int wy = t0r / 2 + a.ka_r0, wx = t0c / 2 + a.ka_c0 - a.d_c;
    const int rhi = min(max(a.nr - wy, 0), G::BR), chi = min(max(a.nc - wx, 0), G::BC);
    const int side = G::BC - chi, below = G::BR - rhi;
    const bool wrap = a.wrap && (side > 0 || below > 0);
    float rv[NRS], bv[NBS];
    if (wrap) {
#pragma unroll
      for (int u = 0; u < NRS; ++u) {  // right strip: rows [0, rhi), columns [chi, BC)
        const int i = tid + u * kNT, bb = i / RS, rem = i - bb * RS, rr = rem / kWrapCols, k = rem - rr * kWrapCols;
        rv[u] = 0.0f;
        if (i < 4 * RS && rr < rhi && k < side) {
          const float* src = bb == 0 ? a.band[0] : (bb == 1 ? a.band[1] : (bb == 2 ? a.band[2] : a.band[3]));
          rv[u] = __ldg(src + (size_t)(wy + rr) * a.band_pitch + k);
        }
      }
#pragma unroll
      for (int u = 0; u < NBS; ++u) {  // bottom strip: rows [rhi, BR), all columns
        const int i = tid + u * kNT, bb = i / BS, rem = i - bb * BS, r2 = rem / G::BC, cc = rem - r2 * G::BC;
        bv[u] = 0.0f;
        if (i < 4 * BS && r2 < below) {
          const float* src = bb == 0 ? a.band[0] : (bb == 1 ? a.band[1] : (bb == 2 ? a.band[2] : a.band[3]));
          const int col = wx + cc >= a.nc ? wx + cc - a.nc : wx + cc;
          bv[u] = __ldg(src + (size_t)r2 * a.band_pitch + col);
        }
      }
    }
    bool ok = mbar_wait(&bar[b], (phase >> b) & 1);
    if (ok) {
      phase ^= 1u << b;
      pending &= ~(1u << b);
    }
    if (!__syncthreads_and(ok)) {
      if (tid == 0) record_status(a.status, ADJWT_ERR_TIMEOUT);
      for (int bb = 0; bb < 2; ++bb)
        if (pending & (1u << bb)) mbar_wait(&bar[bb], (phase >> bb) & 1);
      if (tid == 0) bulk_wait_all();
      return;
    }
    float* S = buf0 + b * G::BUF;
    if (wrap) {
#pragma unroll
      for (int u = 0; u < NRS; ++u) {
        const int i = tid + u * kNT, bb = i / RS, rem = i - bb * RS, rr = rem / kWrapCols, k = rem - rr * kWrapCols;
        if (i < 4 * RS && rr < rhi && k < side) S[bb * G::BAND + rr * G::BC + chi + k] = rv[u];
      }
#pragma unroll
      for (int u = 0; u < NBS; ++u) {
        const int i = tid + u * kNT, bb = i / BS, rem = i - bb * BS, r2 = rem / G::BC, cc = rem - r2 * G::BC;
        if (i < 4 * BS && r2 < below) S[bb * G::BAND + (rhi + r2) * G::BC + cc] = bv[u];
      }
      __syncthreads();
    }
    // column pass: item = (hb, row block, coefficient column)
    for (int item = tid; item < 2 * 2 * a.nk_c; item += kNT) {
      const int hb = item >= 2 * a.nk_c ? 1 : 0;
      const int rem = item - hb * 2 * a.nk_c;
      const int rb = rem >= a.nk_c ? 1 : 0, ll = rem - rb * a.nk_c;
      const float* s0 = S + (2 * hb) * G::BAND + (kP * rb) * G::BC + a.d_c + ll;
      const float* s1 = s0 + G::BAND;
      float c0[G::NC], c1[G::NC], out[2 * kP];
#pragma unroll
      for (int j = 0; j < G::NC; ++j) {
        c0[j] = s0[j * G::BC];
        c1[j] = s1[j * G::BC];
      }
      if (a.phi_r)
        pairs<L, 1>(c0, c1, a, out);
      else
        pairs<L, 0>(c0, c1, a, out);
      float* g = Gf + (hb * kTH + 2 * kP * rb) * G::GP + ll;
#pragma unroll
      for (int o = 0; o < 2 * kP; ++o) g[o * G::GP] = out[o];
    }
    __syncthreads();
    // the column pass has consumed this staging buffer; the other one (whose
    // staged output tile the previous tile's bulk stores have read) takes the
    // next tile's copies
    if (t + gridDim.x < a.ntiles) {
      if (tid == 0) bulk_wait_read();
      issue(t + gridDim.x, b ^ 1);
    }
    float* St = buf0 + (b ? G::OUT1 : G::OUT0);
    // row pass: warp = 16-pixel block, lane = row; results staged for the bulk stores
    {
      const int warp = tid >> 5, r = tid & 31;
      if (warp < kTW / (2 * kP)) {
        const float* g0 = Gf + r * G::GP + kP * warp;
        const float* g1 = g0 + kTH * G::GP;
        float c0[G::NC], c1[G::NC], out[2 * kP];
#pragma unroll
        for (int j = 0; j < G::NC; ++j) {
          c0[j] = g0[j];
          c1[j] = g1[j];
        }
        if (a.phi_c)
          pairs<L, 1>(c0, c1, a, out);
        else
          pairs<L, 0>(c0, c1, a, out);
        // 16-byte chunk c of row r of box x/32 at chunk position c xor (r mod 8):
        // a quarter warp (8 consecutive rows, same chunk) hits 8 distinct bank groups
#pragma unroll
        for (int q = 0; q < kP / 2; ++q) {
          const int col = 2 * kP * warp + 4 * q;
          float* d = St + (col >> 5) * (kTH * 32) + r * 32 + ((((col >> 2) & 7) ^ (r & 7)) << 2);
          *reinterpret_cast<float4*>(d) = make_float4(out[4 * q], out[4 * q + 1], out[4 * q + 2], out[4 * q + 3]);
        }
      }
    }
    fence_proxy_async();  // the staged tile -> the bulk stores
    __syncthreads();      // also: Gf is rewritten next
    if (tid == 0) {
#pragma unroll
      for (int bx = 0; bx < kTW / 32; ++bx) tma_store_2d(&mo, St + bx * (kTH * 32), t0c + 32 * bx, t0r);
      bulk_commit();
    }
  }
  if (tid == 0) bulk_wait_all();  // the output is in global memory before the CTA exits
}

// Interior tile range [lo, hi) along one axis (tile size T): tiles whose
// outputs need no mirrored copy, no weight, and whose coefficients lie inside
// the band.
void interior_range(int N, int n, int T, int mode, int L, bool weighted, int* lo, int* hi) {
  if (mode == kZero || mode == kPer) {  // zero fill / wrap fill cover the band edges
    *lo = 0;
    *hi = N / T;
    return;
  }
  const int Lp = L - 1, off = mode == kPer ? Lp : 2 * Lp;
  const bool sym = mode == kSym;
  const int guard = (weighted || sym) ? Lp : 0;
  *lo = 0;
  *hi = 0;
  bool found = false;
  for (int t = 0; (t + 1) * T <= N; ++t) {
    const int t0 = t * T;
    bool ok = t0 >= guard && t0 + T <= N - guard;
    if (sym) ok = ok && t0 >= Lp && t0 + T <= N - Lp;
    const int phi = (t0 + off - 1) & 1;
    const int Kb = (t0 + off - 1) >> 1;  // t0 + off - 1 >= 0
    const int ka = Kb - (L / 2 - 1), nk = T / 2 + L / 2 - 1 + phi;
    ok = ok && ka >= 0 && ka + nk <= n;
    if (ok && !found) {
      *lo = t;
      found = true;
    }
    if (ok) *hi = t + 1;
    if (!ok && found) break;
  }
}

template <int L>
int launch_l(const SynTmaArgs& a, const CUtensorMap (&maps)[5], cudaStream_t s, int level, int ctas) {
  using G = SG<L>;
  const size_t smem = G::smem_bytes();
  ADJWT_CUDA_CHECK(set_smem(k_synth_tma<L>, smem));
  static int occ = 0;
  if (!occ) {
    int v = 0;
    ADJWT_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_synth_tma<L>, kNT, smem));
    occ = std::max(v, 1);
  }
  const int grid = std::min(a.ntiles, sm_count() * (ctas > 0 ? std::min(ctas, occ) : occ));
  ADJWT_TRACED("wt_synth_tma", level, s,
               pdl_launch(k_synth_tma<L>, grid, kNT, smem, s, maps[0], maps[1], maps[2], maps[3], maps[4], a));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  return ADJWT_OK;
}

}  // namespace

// Pixel rectangle [r0, r1) x [c0, c1) of level j's output reconstructed by the
// TMA kernel (empty when the level is small); the tiled kernel skips it.
void synth_tma_rect(const adjwt_wt_plan* p, int j, int* r0, int* r1, int* c0, int* c1) {
  *r0 = *r1 = *c0 = *c1 = 0;
  if (p->tma_off[0][j - 1]) return;
  const Level& L = p->lv[j - 1];
  if (L.generic_synth || L.ax[0].N < 256 || L.ax[1].N < 512) return;
  const bool weighted = L.ax[0].winv != nullptr || p->bc == kPpd;
  int ylo, yhi, xlo, xhi;
  interior_range(L.ax[0].N, L.ax[0].n, kTH, p->bc, p->fb.L, weighted, &ylo, &yhi);
  interior_range(L.ax[1].N, L.ax[1].n, kTW, p->bc, p->fb.L, weighted, &xlo, &xhi);
  if (yhi - ylo < 2 || xhi - xlo < 1) return;
  // sharing a level with the tiled kernel pays only on large levels: the
  // tiled kernel's border tiles cost about as much as the whole of a small one
  const bool whole = ylo == 0 && xlo == 0 && yhi * kTH == L.ax[0].N && xhi * kTW == L.ax[1].N;
  if (!whole && (L.ax[0].N < kSplitMin || L.ax[1].N < kSplitMin)) return;
  *r0 = ylo * kTH;
  *r1 = yhi * kTH;
  *c0 = xlo * kTW;
  *c1 = xhi * kTW;
}

int launch_synth_tma(const adjwt_wt_plan* p, int j, const float* const band[4], float* out, int out_pitch,
                     cudaStream_t s) {
  int r0, r1, c0, c1;
  synth_tma_rect(p, j, &r0, &r1, &c0, &c1);
  if (r1 <= r0 || c1 <= c0) return ADJWT_OK;
  const Level& L = p->lv[j - 1];
  const int Lf = p->fb.L, Lp = Lf - 1, off = p->bc == kPer ? Lp : 2 * Lp;
  SynTmaArgs a{};
  a.out = out;
  a.out_pitch = out_pitch;
  // tiles start at even t0, so phi and ka - t0/2 are the same for every tile
  a.phi_r = a.phi_c = (off - 1) & 1;
  a.ka_r0 = a.ka_c0 = (off - 1 - a.phi_r) / 2 - (Lf / 2 - 1);
  a.d_c = a.ka_c0 & 3;  // t0c / 2 is a multiple of 4
  a.nk_c = kTW / 2 + Lf / 2 - 1 + a.phi_c;
  a.ty0 = r0 / kTH;
  a.tx0 = c0 / kTW;
  a.ntx = (c1 - c0) / kTW;
  a.ntiles = a.ntx * ((r1 - r0) / kTH);
  a.wrap = p->bc == kPer;
  // box origin of the last full tile (its overhang past the band end is the largest)
  const int last_r = (r1 - kTH) / 2 + a.ka_r0, last_c = (c1 - kTW) / 2 + a.ka_c0 - a.d_c;
  a.nr = L.ax[0].n;
  a.nc = L.ax[1].n;
  a.band_pitch = L.band_pitch;
  for (int b = 0; b < 4; ++b) a.band[b] = band[b];
  a.status = device_status_ptr();
  for (int t = 0; t < Lf; ++t) {
    a.g[0][t] = static_cast<float>(p->fb.rec_lo[t]);
    a.g[1][t] = static_cast<float>(p->fb.rec_hi[t]);
  }
  return [&]() -> int {
    switch (Lf) {
#define ADJWT_L(LL)                                                                                     \
  case LL: {                                                                                            \
    if (a.wrap && (last_r + SG<LL>::BR - L.ax[0].n > kWrapRows || last_c + SG<LL>::BC - L.ax[1].n > kWrapCols)) \
      return fail(ADJWT_ERR_SHAPE, "TMA reconstruction: periodic overhang above the staged bound");     \
    CUtensorMap maps[5];                                                                                \
    for (int b = 0; b < 4; ++b) {                                                                       \
      int rc = make_tmap_2d_f32(&maps[b], band[b], L.ax[0].n, L.ax[1].n, L.band_pitch, SG<LL>::BR,      \
                                SG<LL>::BC);                                                            \
      if (rc) return rc;                                                                                \
    }                                                                                                   \
    /* the output: 32 x 32 boxes, 128-byte swizzle */                                                   \
    int rc = make_tmap_2d_f32_sw(&maps[4], out, L.ax[0].N, out_pitch, out_pitch, kTH, 32, true);        \
    if (rc) return rc;                                                                                  \
    return launch_l<LL>(a, maps, s, j, p->tma_ctas[0][j - 1]);                                          \
  }
      ADJWT_L(2) ADJWT_L(4) ADJWT_L(8) ADJWT_L(10)
#undef ADJWT_L
      default:
        return fail(ADJWT_ERR_INVALID_ARG, "unsupported filter length");
    }
  }();
}


// ===================================================================== analysis
// Persistent TMA-staged W^* (+ the FISTA prox) / W^dagger for every tile of
// a level.  The TMA unit's zero fill is the zero extension; a border tile's
// window is completed after the copy from the extension map and the 1/c
// weights (border_prefetch / border_apply); border tiles are walked first
// (border_first_tile), so that no CTA takes two of them.
// A tile is kAR x kAC coefficients of each band; its input window is
// (2 kAR + L - 2) x (2 kAC + L - 2) samples of the extended signal, staged by
// the TMA unit into one of two buffers while the previous tile is filtered:
//   column pass: a thread filters 8 coefficient rows of one window column
//                with both analysis filters from a register window;
//   row pass:    lanes on (vertical filter, coefficient row), a warp per
//                8-coefficient block; both horizontal filters, then the
//                plain result or the prox epilogue.  Every output band tile
//                (16 x 64) is staged as two 16 x 32 boxes under the 128-byte
//                swizzle and written by TMA stores (rows past the band and
//                columns past the pitch are clipped; pad columns are staged
//                as zero); the prox state y, x of the tile comes in the same
//                way, one tile ahead, and is updated in place.
namespace {

constexpr int kAR = 16;    // coefficient rows per tile
constexpr int kAC = 64;    // coefficient columns per tile
constexpr int kAP = 8;     // outputs per thread and pass

template <int L>
struct AG {
  static constexpr int ER = 2 * kAR + L - 2;      // window rows
  static constexpr int EC = 2 * kAC + L - 2;      // window columns
  static constexpr int BC = up4(EC + 3);          // box columns (16-byte start slack)
  static constexpr int BUF = up32(ER * BC);
  static constexpr int NW = 2 * kAP + L - 2;      // register window per thread
  static constexpr int VP = EC | 1;               // odd pitch of the column-pass output
  // Output tiles (and, with the prox, the state y and x of the prox bands)
  // are staged as 16 x 32 boxes of 128-byte rows under the 128-byte swizzle:
  // the outputs of a band in the window buffer the column pass has consumed
  // (from a 1024-byte boundary inside it), y and x of every prox band in P.
  static constexpr int OUT0 = 0;                        // staging of buffer 0 (floats, 256-float aligned)
  static constexpr int OUT1 = (BUF + 255) / 256 * 256;  // staging of buffer 1
  static constexpr int V0 = 2 * BUF;
  static constexpr int P0 = (V0 + 2 * kAR * VP + 255) / 256 * 256;
  static_assert(OUT1 + 4 * 2 * kAR * 32 <= 2 * BUF, "four staged bands fit in window buffer 1");
  static_assert(4 * 2 * kAR * 32 <= BUF, "four staged bands fit in window buffer 0");
  static constexpr size_t smem_bytes(bool prox) {
    return 1024 + (size_t)(prox ? P0 + 8 * 2 * kAR * 32 : V0 + 2 * kAR * VP) * 4;
  }
};

constexpr int kOB = kAR * 32;   // floats per staged 16 x 32 box
constexpr int kOBand = 2 * kOB; // one band's 16 x 64 tile

// Float offset of coefficient (r, c), c < 64, in a band tile staged as two
// 16 x 32 boxes under the 128-byte swizzle (16-byte chunk c/4 of row r at
// chunk position (c/4) xor (r mod 8)).  A quarter warp on 8 consecutive rows
// reading the same 16-byte column chunk hits 8 distinct bank groups.
__device__ __forceinline__ int sw_off(int r, int c) {
  return (c >> 5) * kOB + r * 32 + ((((c >> 2) & 7) ^ (r & 7)) << 2) + (c & 3);
}

// Tensor maps of the output bands (16 x 32 boxes, 128-byte swizzle) over the
// band_rows x out_pitch bands: for band i, m[2 i] is y of a prox band or the
// plain destination, m[2 i + 1] is x of a prox band.
struct AnaOutMaps {
  CUtensorMap m[8];
};

struct AnaTmaArgs {
  int sh;                 // image index of extended sample e is e - sh
  int d_c;                // window column start minus its 16-byte-aligned start
  int ty0, tx0, ntx, ntiles;
  // tiles whose window needs no border completion: rows [ir0, ir1), columns
  // [ic0, ic1) (tile units; nty tile rows).  The others are numbered first.
  int nty, ir0, ir1, ic0, ic1;
  int out_pitch;
  // border tiles: the level input and its extension (fix = 0 under ZERO,
  // where the box's zero fill is the whole extension)
  const float* in;
  int in_pitch, Nr, Nc, nr, nc, mode, fix;
  const float* winv_r;    // 1/c weights of W^* (null for W^dagger and PER / ZERO)
  const float* winv_c;
  float* dst[4];          // plain destinations (LL, LH, HL, HH)
  float* px[4];           // prox state (non-null => prox band)
  float* py[4];
  float step, thresh, beta;
  const double* beta_dev; // non-null: beta from device memory
  double* l1;             // per-CTA partials of |x| (null = skip)
  int* status;
  float flo[kMaxTaps], fhi[kMaxTaps];
};

// Border tiles.  The box holds img[e - sh] for every window cell whose image
// index lies inside the image and zero elsewhere.  What the extension needs
// beyond that:
//   * off-image cells under the symmetric / periodic extensions hold a mirror
//     or wrap copy (zero outside the extended signal).  A half-point mirror
//     of a border window lies inside the same window (for levels of the TMA
//     size), so those cells are copied within shared memory; wrap copies
//     (and mirrors outside the window) are fetched from the image into
//     registers while the copy is in flight;
//   * every cell then takes the weights 1/c of its source row and column
//     (W^*'s weighted extension (E^dagger)^*, Eq. 2), from per-row and
//     per-column tables built before the copy has landed.
// Off-image cells are enumerated as strips (rows above / below the image at
// full width, then the columns beside it on the other rows).
struct AnaBorder {
  int e0r, e0c;             // extended coordinates of window row / column 0
  int rlo, rhi, clo, chi;   // in-image window rows [rlo, rhi), columns [clo, chi)
  int side, ntop, nbot, total;
  bool any;                 // anything to do for this tile (uniform)
  bool weighted;            // some weight differs from 1
};

// Per window row (first ER entries) and column (next EC): the source image
// index (-1: zero), the window index of the source when the window holds it
// (-1: not held), and the weight 1/c of the source (1 without weights).
template <int L>
struct BorderTables {
  int img[AG<L>::ER + AG<L>::EC];
  int win[AG<L>::ER + AG<L>::EC];
  float w[AG<L>::ER + AG<L>::EC];
};

template <int L>
__device__ __forceinline__ AnaBorder ana_border(const AnaTmaArgs& a, int k0, int l0) {
  using G = AG<L>;
  constexpr int Lp = L - 1;
  AnaBorder b;
  b.e0r = 2 * k0 + 1 - Lp;
  b.e0c = 2 * l0 + 1 - Lp;
  const int xr = b.e0r - a.sh, xc = b.e0c - a.sh;  // image index of window row / column 0
  b.rlo = min(max(-xr, 0), G::ER);
  b.rhi = min(max(a.Nr - xr, b.rlo), G::ER);
  b.clo = min(max(-xc, 0), G::EC);
  b.chi = min(max(a.Nc - xc, b.clo), G::EC);
  b.side = b.clo + (G::EC - b.chi);
  b.ntop = b.rlo * G::EC;
  b.nbot = (G::ER - b.rhi) * G::EC;
  b.total = a.fix ? b.ntop + b.nbot + (b.rhi - b.rlo) * b.side : 0;
  const bool wr = a.winv_r && (xr < Lp || xr + G::ER > a.Nr - Lp);
  const bool wc = a.winv_c && (xc < Lp || xc + G::EC > a.Nc - Lp);
  b.weighted = wr || wc;
  b.any = b.total > 0 || b.weighted;
  return b;
}

// window cell (row * EC + col) of off-image cell i < total
template <int L>
__device__ __forceinline__ int border_cell(const AnaBorder& b, int i) {
  using G = AG<L>;
  if (i < b.ntop) return i;
  if (i < b.ntop + b.nbot) return b.rhi * G::EC + (i - b.ntop);
  const int j = i - b.ntop - b.nbot, rr = j / b.side, k = j - rr * b.side;
  return (b.rlo + rr) * G::EC + (k < b.clo ? k : b.chi + (k - b.clo));
}

// source image index of extended coordinate e (-1: zero)
template <int L>
__device__ __forceinline__ int ana_src(const AnaTmaArgs& a, int e, int N) {
  constexpr int Lp = L - 1;
  if (a.mode == kPer) return pos_mod(e, N);
  return (e >= 0 && e < N + 2 * Lp) ? ext_src(e - Lp, N, a.mode) : -1;
}

template <int L>
__device__ __forceinline__ void border_tables(const AnaTmaArgs& a, const AnaBorder& b, BorderTables<L>& t) {
  using G = AG<L>;
  for (int i = threadIdx.x; i < G::ER + G::EC; i += kNT) {
    const bool row = i < G::ER;
    const int u = row ? i : i - G::ER;
    const int N = row ? a.Nr : a.Nc, E = row ? G::ER : G::EC;
    const int x0 = (row ? b.e0r : b.e0c) - a.sh;
    const int src = ana_src<L>(a, x0 + u + a.sh, N);
    const float* winv = row ? a.winv_r : a.winv_c;
    const int wi = src >= 0 ? src - x0 : -1;
    t.img[i] = src;
    t.win[i] = (wi >= 0 && wi < E) ? wi : -1;
    t.w[i] = (src >= 0 && winv) ? __ldg(winv + src) : 1.0f;
  }
}

constexpr int kFixRegs = 10;  // far off-image cells per thread fetched before the copy has landed

// far source of an off-image cell (not held by the window): straight from the image, unweighted
template <int L>
__device__ __forceinline__ float border_far(const AnaTmaArgs& a, const AnaBorder& b, int cell) {
  using G = AG<L>;
  const int r = cell / G::EC, c = cell - r * G::EC;
  const int sr = ana_src<L>(a, b.e0r + r, a.Nr), sc = ana_src<L>(a, b.e0c + c, a.Nc);
  return (sr >= 0 && sc >= 0 && in_bounds(a.status, sr < a.Nr && sc < a.Nc))
             ? __ldg(a.in + (size_t)sr * a.in_pitch + sc)
             : 0.0f;
}

// Before the copy has landed: the tables, and (periodic extensions) the far
// off-image cells into registers.
// The border code is out of line: most tiles never run it, and keeping it out
// of the tile loop's instruction stream cut the kernel's instruction-fetch
// stalls (W^* + prox level 1 at 2048^2: 30.2 -> 28.8 us).
template <int L>
__device__ __noinline__ void border_prefetch(const AnaTmaArgs& a, const AnaBorder& b, BorderTables<L>& t,
                                                float (&fv)[kFixRegs]) {
  border_tables<L>(a, b, t);
  if (a.mode != kSym) {
#pragma unroll
    for (int u = 0; u < kFixRegs; ++u) {
      const int i = threadIdx.x + u * kNT;
      fv[u] = i < b.total ? border_far<L>(a, b, border_cell<L>(b, i)) : 0.0f;
    }
  }
}

// After the copy (and a block barrier, so the tables are visible): the
// off-image cells, then the weights.  Ends with a block barrier.
template <int L>
__device__ __noinline__ void border_apply(const AnaTmaArgs& a, const AnaBorder& b, const BorderTables<L>& t,
                                             const float (&fv)[kFixRegs], float* S) {
  using G = AG<L>;
  if (a.mode == kSym) {
    // mirror copies from in-image cells of the same window (never off-image
    // themselves, so the copies can run in any order)
    for (int i = threadIdx.x; i < b.total; i += kNT) {
      const int cell = border_cell<L>(b, i), r = cell / G::EC, c = cell - r * G::EC;
      const int wr = t.win[r], wc = t.win[G::ER + c];
      float v = 0.0f;
      if (wr >= 0 && wc >= 0) {
        if (in_bounds(a.status, wr < G::ER && wc < G::EC)) v = S[wr * G::BC + wc];
      } else {
        const int sr = t.img[r], sc = t.img[G::ER + c];
        if (sr >= 0 && sc >= 0 && in_bounds(a.status, sr < a.Nr && sc < a.Nc))
          v = __ldg(a.in + (size_t)sr * a.in_pitch + sc);
      }
      S[r * G::BC + c] = v;
    }
  } else {
#pragma unroll
    for (int u = 0; u < kFixRegs; ++u) {
      const int i = threadIdx.x + u * kNT;
      if (i < b.total) {
        const int c = border_cell<L>(b, i), r = c / G::EC;
        S[r * G::BC + (c - r * G::EC)] = fv[u];
      }
    }
    for (int i = threadIdx.x + kFixRegs * kNT; i < b.total; i += kNT) {  // larger overhangs
      const int c = border_cell<L>(b, i), r = c / G::EC;
      S[r * G::BC + (c - r * G::EC)] = border_far<L>(a, b, c);
    }
  }
  if (b.weighted) {
    __syncthreads();  // every cell holds its unweighted source value
    for (int i = threadIdx.x; i < G::ER * G::EC; i += kNT) {
      const int r = i / G::EC, c = i - r * G::EC;
      const float w = t.w[r] * t.w[G::ER + c];
      if (w != 1.0f) S[r * G::BC + c] *= w;
    }
  }
  fence_proxy_async();  // these generic writes come before the TMA unit's next write into the buffer
  __syncthreads();
}

template <int L, bool PROX>
__global__ void __launch_bounds__(kNT, PROX ? 2 : 3)
    k_ana_tma(const __grid_constant__ CUtensorMap map, const __grid_constant__ AnaOutMaps om, const AnaTmaArgs a) {
  pdl_entry();
  using G = AG<L>;
  constexpr int Lp = L - 1;
  extern __shared__ unsigned char dyn[];
  __shared__ uint64_t bar[2];
  __shared__ uint64_t pbar;  // prox state of the current tile
  __shared__ double red[kNT / 32];
  __shared__ BorderTables<L> tabs;  // border tiles
  float* buf0 = reinterpret_cast<float*>(dyn + ((1024 - (smem_u32(dyn) & 1023)) & 1023));
  float* V = buf0 + G::V0;  // [2][kAR][VP]
  float* P = buf0 + G::P0;  // prox: y, x of band i at P + (2 i) kOBand, P + (2 i + 1) kOBand
  const int tid = threadIdx.x;

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init(&pbar, 1);
    fence_mbar_init();
  }
  __syncthreads();

  uint32_t phase = 0, pending = 0, pphase = 0, ppending = 0;
  // Tile t: the border tiles (whose windows need completing, the slow ones)
  // come first, so that every CTA takes at most one and starts with it; then
  // the interior tiles row by row.
  auto tile_origin = [&](int t, int& k0, int& l0) {
    int ty, tx;
    border_first_tile(t, a.ntx, a.nty, a.ir0, a.ir1, a.ic0, a.ic1, &ty, &tx);
    k0 = (a.ty0 + ty) * kAR;
    l0 = (a.tx0 + tx) * kAC;
  };
  auto issue = [&](int t, int b) {
    int k0, l0;
    tile_origin(t, k0, l0);
    if (tid == 0) {
      fence_proxy_async();
      mbar_arrive_expect_tx(&bar[b], G::ER * G::BC * 4);
      tma_load_2d(buf0 + b * G::BUF, &map, &bar[b], 2 * l0 + 1 - Lp - a.sh - a.d_c, 2 * k0 + 1 - Lp - a.sh);
    }
    pending |= 1u << b;
  };
  // prox variant: y and x of every prox band of tile t into P (two boxes each;
  // boxes past the band read as zero)
  int nprox = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) nprox += a.px[i] != nullptr;
  auto issue_prox = [&](int t) {
    int k0, l0;
    tile_origin(t, k0, l0);
    if (tid == 0) {
      mbar_arrive_expect_tx(&pbar, nprox * 2 * kOBand * 4);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (!a.px[i]) continue;
#pragma unroll
        for (int bx = 0; bx < 2; ++bx) {
          tma_load_2d(P + 2 * i * kOBand + bx * kOB, &om.m[2 * i], &pbar, l0 + 32 * bx, k0);
          tma_load_2d(P + (2 * i + 1) * kOBand + bx * kOB, &om.m[2 * i + 1], &pbar, l0 + 32 * bx, k0);
        }
      }
    }
    ppending = 1;
  };
  auto drain = [&]() {
    for (int bb = 0; bb < 2; ++bb)
      if (pending & (1u << bb)) mbar_wait(&bar[bb], (phase >> bb) & 1);
    if (PROX && ppending) mbar_wait(&pbar, pphase & 1);
    if (tid == 0) bulk_wait_all();
  };

  float l1 = 0.0f;
  const float beta = PROX && a.beta_dev ? static_cast<float>(*a.beta_dev) : a.beta;
  // row-pass thread: (vertical filter f, coefficient row kk), 8-coefficient block = warp
  const int warp = tid >> 5, lane = tid & 31, f = lane >> 4, kk = lane & 15;
  const bool rower = warp < kAC / kAP;
  int t = blockIdx.x, b = 0;
  if (t < a.ntiles) {
    issue(t, 0);
    if (PROX) issue_prox(t);
  }
  for (; t < a.ntiles; t += gridDim.x, b ^= 1) {
    int k0, l0;
    tile_origin(t, k0, l0);
    const bool rvalid = k0 + kk < a.nr;     // the last row tile may be partial
    const int lbase = l0 + kAP * warp;      // and the last column tile
    // border tile: tables (and far off-image cells) fetched while the copy is in flight
    const AnaBorder bd = ana_border<L>(a, k0, l0);
    float fv[kFixRegs];
    if (bd.any) border_prefetch<L>(a, bd, tabs, fv);
    bool ok = mbar_wait(&bar[b], (phase >> b) & 1);
    if (ok) {
      phase ^= 1u << b;
      pending &= ~(1u << b);
    }
    if (!__syncthreads_and(ok)) {
      if (tid == 0) record_status(a.status, ADJWT_ERR_TIMEOUT);
      drain();
      return;
    }
    // every thread is past the previous tile: the other window buffer (whose
    // staged outputs the bulk stores have read) takes the next tile's copy
    if (t + gridDim.x < a.ntiles) {
      if (tid == 0) bulk_wait_read();
      issue(t + gridDim.x, b ^ 1);
    }
    if (bd.any) border_apply<L>(a, bd, tabs, fv, buf0 + b * G::BUF + a.d_c);
    const float* S = buf0 + b * G::BUF + a.d_c;
    // column pass: V[f][kk][ec] = sum_t f[t] T[2 kk + L' - t][ec]
    for (int item = tid; item < 2 * G::EC; item += kNT) {
      const int rb = item >= G::EC ? 1 : 0, ec = item - rb * G::EC;
      const float* src = S + 2 * kAP * rb * G::BC + ec;
      float w[G::NW];
#pragma unroll
      for (int j = 0; j < G::NW; ++j) w[j] = src[j * G::BC];
      float* v0 = V + (kAP * rb) * G::VP + ec;
      float* v1 = v0 + kAR * G::VP;
#pragma unroll
      for (int p = 0; p < kAP; ++p) {
        float lo = 0.0f, hi = 0.0f;
#pragma unroll
        for (int q = 0; q < L; ++q) {
          lo = fmaf(a.flo[q], w[2 * p + Lp - q], lo);
          hi = fmaf(a.fhi[q], w[2 * p + Lp - q], hi);
        }
        v0[p * G::VP] = lo;
        v1[p * G::VP] = hi;
      }
    }
    bool pok = true;
    if (PROX && tid == 0) pok = mbar_wait(&pbar, pphase & 1);
    if (!__syncthreads_and(pok)) {
      if (tid == 0) record_status(a.status, ADJWT_ERR_TIMEOUT);
      drain();
      return;
    }
    if (PROX) {
      pphase ^= 1;
      ppending = 0;
    }
    // outputs staged in this tile's window buffer (the column pass has consumed it)
    float* D = buf0 + (b ? G::OUT1 : G::OUT0);
    // row pass + prox epilogue into the staged tiles
    if (rower) {
      const float* src = V + (f * kAR + kk) * G::VP + 2 * kAP * warp;
      float w[G::NW];
#pragma unroll
      for (int j = 0; j < G::NW; ++j) w[j] = src[j];
      float res[2][kAP];
#pragma unroll
      for (int p = 0; p < kAP; ++p) {
        float lo = 0.0f, hi = 0.0f;
#pragma unroll
        for (int q = 0; q < L; ++q) {
          lo = fmaf(a.flo[q], w[2 * p + Lp - q], lo);
          hi = fmaf(a.fhi[q], w[2 * p + Lp - q], hi);
        }
        res[0][p] = lo;
        res[1][p] = hi;
      }
      // pad columns (band index >= nc, inside the pitch) are written as zero
#pragma unroll
      for (int p = 0; p < kAP; ++p)
        if (lbase + p >= a.nc) res[0][p] = res[1][p] = 0.0f;
      const int o0 = sw_off(kk, kAP * warp), o1 = sw_off(kk, kAP * warp + 4);
#pragma unroll
      for (int hb = 0; hb < 2; ++hb) {
        const int band = f + 2 * hb;
        if (PROX && a.px[band]) {
          float* Y = P + 2 * band * kOBand;
          float* X = Y + kOBand;
          const float4 y4[2] = {*reinterpret_cast<const float4*>(Y + o0), *reinterpret_cast<const float4*>(Y + o1)};
          const float4 x4[2] = {*reinterpret_cast<const float4*>(X + o0), *reinterpret_cast<const float4*>(X + o1)};
          const float yv[kAP] = {y4[0].x, y4[0].y, y4[0].z, y4[0].w, y4[1].x, y4[1].y, y4[1].z, y4[1].w};
          const float xv[kAP] = {x4[0].x, x4[0].y, x4[0].z, x4[0].w, x4[1].x, x4[1].y, x4[1].z, x4[1].w};
          float xn[kAP], yn[kAP];
#pragma unroll
          for (int p = 0; p < kAP; ++p) {
            const float v = yv[p] - a.step * res[hb][p];
            const float mag = fabsf(v) - a.thresh;
            float x = mag > 0.0f ? copysignf(mag, v) : 0.0f;
            float y = fmaf(beta, x - xv[p], x);
            if (lbase + p >= a.nc) x = y = 0.0f;
            xn[p] = x;
            yn[p] = y;
            if (a.l1 && rvalid) l1 += fabsf(x);
          }
          *reinterpret_cast<float4*>(X + o0) = make_float4(xn[0], xn[1], xn[2], xn[3]);
          *reinterpret_cast<float4*>(X + o1) = make_float4(xn[4], xn[5], xn[6], xn[7]);
          *reinterpret_cast<float4*>(Y + o0) = make_float4(yn[0], yn[1], yn[2], yn[3]);
          *reinterpret_cast<float4*>(Y + o1) = make_float4(yn[4], yn[5], yn[6], yn[7]);
        } else if (a.dst[band]) {
          float* Db = D + band * kOBand;
          *reinterpret_cast<float4*>(Db + o0) = make_float4(res[hb][0], res[hb][1], res[hb][2], res[hb][3]);
          *reinterpret_cast<float4*>(Db + o1) = make_float4(res[hb][4], res[hb][5], res[hb][6], res[hb][7]);
        }
      }
    }
    fence_proxy_async();  // the staged tiles -> the bulk stores
    __syncthreads();
    if (tid == 0) {
      // rows past the band and columns past the pitch are not written
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const bool prox = PROX && a.px[i];
        if (!prox && !a.dst[i]) continue;
#pragma unroll
        for (int bx = 0; bx < 2; ++bx) {
          if (l0 + 32 * bx >= a.out_pitch) continue;
          if (prox) {
            tma_store_2d(&om.m[2 * i], P + 2 * i * kOBand + bx * kOB, l0 + 32 * bx, k0);
            tma_store_2d(&om.m[2 * i + 1], P + (2 * i + 1) * kOBand + bx * kOB, l0 + 32 * bx, k0);
          } else {
            tma_store_2d(&om.m[2 * i], D + i * kOBand + bx * kOB, l0 + 32 * bx, k0);
          }
        }
      }
      bulk_commit();
    }
    // the next tile's prox state goes into P once the stores have read it
    if (PROX && t + gridDim.x < a.ntiles) {
      if (tid == 0) bulk_wait_read();
      issue_prox(t + gridDim.x);
    }
  }
  if (tid == 0) bulk_wait_all();  // the staged outputs are in global memory before the CTA exits
  if (a.l1) {
    const double tot = block_sum<kNT>((double)l1, red);
    if (tid == 0) a.l1[blockIdx.x] = tot;
  }
}

// Full coefficient tiles [lo, hi) (tile size T) along one axis whose input
// window stays inside [guard, N - guard) (any window under ZERO).
void ana_range(int N, int n, int T, int mode, int L, bool weighted, int* lo, int* hi) {
  const int Lp = L - 1, sh = mode == kPer ? 0 : Lp, E = 2 * T + L - 2;
  const int guard = weighted ? Lp : 0;
  *lo = *hi = 0;
  bool found = false;
  for (int t = 0; (t + 1) * T <= n; ++t) {
    const int first = 2 * t * T + 1 - Lp - sh, last = first + E - 1;
    const bool ok = mode == kZero || (first >= guard && last < N - guard);
    if (ok && !found) {
      *lo = t;
      found = true;
    }
    if (ok) *hi = t + 1;
    if (!ok && found) break;
  }
}

template <int L, bool PROX>
int launch_ana_lp(const AnaTmaArgs& a, const CUtensorMap& map, const AnaOutMaps& om, cudaStream_t s,
                  const char* name, int level, int ctas, int* ncta) {
  using G = AG<L>;
  const size_t smem = G::smem_bytes(PROX);
  auto kern = k_ana_tma<L, PROX>;
  ADJWT_CUDA_CHECK(set_smem(kern, smem));
  static int occ = 0;
  if (!occ) {
    int v = 0;
    ADJWT_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, kNT, smem));
    occ = std::max(v, 1);
  }
  const int grid = std::min(a.ntiles, sm_count() * (ctas > 0 ? std::min(ctas, occ) : occ));
  *ncta = grid;
  ADJWT_TRACED(name, level, s, pdl_launch(kern, grid, kNT, smem, s, map, om, a));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  return ADJWT_OK;
}

template <int L>
int launch_ana_l(const AnaTmaArgs& a, const CUtensorMap& map, const AnaOutMaps& om, cudaStream_t s,
                 const char* name, int level, int ctas, int* ncta) {
  const bool prox = a.px[0] || a.px[1] || a.px[2] || a.px[3];
  return prox ? launch_ana_lp<L, true>(a, map, om, s, name, level, ctas, ncta)
              : launch_ana_lp<L, false>(a, map, om, s, name, level, ctas, ncta);
}

}  // namespace

// Whether level j of the analysis direction runs on the persistent TMA
// kernel (every tile of the level, border tiles included) rather than the
// tiled kernel: levels of at least 1536 x 1536 unless switched off.
bool ana_tma_level(const adjwt_wt_plan* p, int j, bool prox) {
  if (p->tma_off[prox ? 2 : 1][j - 1]) return false;
  const Level& L = p->lv[j - 1];
  // measured on GB300: below about 1536 x 1536 the tiled kernel is as fast or faster
  return L.ax[0].N >= kSplitMin && L.ax[1].N >= kSplitMin;
}

int launch_ana_tma(const adjwt_wt_plan* p, int j, bool adjoint, const float* in, int in_pitch, float* const dst[4],
                   float* const px[4], float* const py[4], int out_pitch, float step, float thresh, float beta,
                   const double* beta_dev, double* l1, const float* flo, const float* fhi, const char* name,
                   cudaStream_t s, int* ncta) {
  *ncta = 0;
  if (!ana_tma_level(p, j, px[1] != nullptr)) return ADJWT_OK;
  const Level& L = p->lv[j - 1];
  const int Lf = p->fb.L, Lp = Lf - 1;
  AnaTmaArgs a{};
  a.sh = p->bc == kPer ? 0 : Lp;
  const int first_c = 1 - Lp - a.sh;  // window start of column tile 0; tiles add 2 kAC (16-byte multiple)
  a.d_c = ((first_c % 4) + 4) % 4;
  a.ty0 = 0;
  a.tx0 = 0;
  a.ntx = (out_pitch + kAC - 1) / kAC;
  a.nty = (L.ax[0].n + kAR - 1) / kAR;
  a.ntiles = a.ntx * a.nty;
  a.out_pitch = out_pitch;
  a.in = in;
  a.in_pitch = in_pitch;
  a.Nr = L.ax[0].N;
  a.Nc = L.ax[1].N;
  a.nr = L.ax[0].n;
  a.nc = L.ax[1].n;
  a.mode = p->bc;
  a.fix = p->bc != kZero;
  a.winv_r = adjoint ? L.ax[0].winv : nullptr;
  a.winv_c = adjoint ? L.ax[1].winv : nullptr;
  // interior tiles per axis: windows [x, x + E) inside [guard, N - guard)
  // (the test of ana_border; under ZERO without weights every tile)
  auto interior = [&](int N, int ntile, int T, int E, bool weighted, int* lo, int* hi) {
    const int guard = weighted ? Lp : 0;
    *lo = *hi = 0;
    bool found = false;
    for (int t = 0; t < ntile; ++t) {
      const int x = 2 * t * T + 1 - Lp - a.sh;
      const bool in = (!a.fix && !weighted) || (x >= guard && x + E <= N - guard);
      if (in && !found) {
        *lo = t;
        found = true;
      }
      if (in) *hi = t + 1;
    }
  };
  const int ER = 2 * kAR + Lf - 2, EC = 2 * kAC + Lf - 2;
  interior(a.Nr, a.nty, kAR, ER, a.winv_r != nullptr, &a.ir0, &a.ir1);
  interior(a.Nc, a.ntx, kAC, EC, a.winv_c != nullptr, &a.ic0, &a.ic1);
  if (a.ir1 <= a.ir0 || a.ic1 <= a.ic0) a.ir0 = a.ir1 = a.ic0 = a.ic1 = 0;  // no interior tile
  for (int b = 0; b < 4; ++b) {
    a.dst[b] = dst[b];
    a.px[b] = px[b];
    a.py[b] = py[b];
  }
  a.step = step;
  a.thresh = thresh;
  a.beta = beta;
  a.beta_dev = beta_dev;
  a.l1 = l1;
  a.status = device_status_ptr();
  for (int t = 0; t < Lf; ++t) {
    a.flo[t] = flo[t];
    a.fhi[t] = fhi[t];
  }
  // output bands (and prox state) move as 16 x 32 boxes: band_rows x out_pitch tensors
  AnaOutMaps om;
  std::memset(&om, 0, sizeof(om));
  for (int b = 0; b < 4; ++b) {
    float* first = px[b] ? py[b] : dst[b];
    if (first) {
      int rc = make_tmap_2d_f32_sw(&om.m[2 * b], first, L.ax[0].n, out_pitch, out_pitch, kAR, 32, true);
      if (rc) return rc;
    }
    if (px[b]) {
      int rc = make_tmap_2d_f32_sw(&om.m[2 * b + 1], px[b], L.ax[0].n, out_pitch, out_pitch, kAR, 32, true);
      if (rc) return rc;
    }
  }
  switch (Lf) {
#define ADJWT_L(LL)                                                                                        \
  case LL: {                                                                                               \
    CUtensorMap map;                                                                                       \
    int rc = make_tmap_2d_f32(&map, in, L.ax[0].N, L.ax[1].N, in_pitch, AG<LL>::ER, AG<LL>::BC);           \
    if (rc) return rc;                                                                                     \
    return launch_ana_l<LL>(a, map, om, s, name, j, p->tma_ctas[px[1] ? 2 : 1][j - 1], ncta);              \
  }
    ADJWT_L(2) ADJWT_L(4) ADJWT_L(8) ADJWT_L(10)
#undef ADJWT_L
    default:
      return fail(ADJWT_ERR_INVALID_ARG, "unsupported filter length");
  }
}

}  // namespace adjwt
