// Persistent TMA-staged single blur pass: R u (optionally - b, optionally
// with per-CTA 1/2 ||R u - b||^2 partials) or R^* v, for radii up to
// kTmaMaxRadius.  Same operator definitions as blur_kernels.cu.
//
// Output tiles are kTH x kTW.  A CTA walks the tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ... with two staging buffers: while it filters tile
// t, the TMA unit already copies the (kTH + 2R) x (kTW + 2 XA) input window of
// the next tile into the other buffer (XA = R rounded up to 4 floats keeps the
// box start 16-byte aligned).  Windows that leave the image are zero-filled
// by the TMA unit, which is exactly the zero extension; under the symmetric
// and periodic extensions the threads then overwrite the off-image cells of
// such border windows through the extension map, and R^* takes the
// orientation-aware taps there (unless the PSF is palindromic, where flipping
// changes nothing).
//
// Per tile: a vertical pass (a thread filters 16 rows of one column from a
// register window, lanes on consecutive columns) writes an odd-pitch buffer
// T; a horizontal pass (lanes on the 32 rows, a warp per 16-column block)
// produces 16 consecutive outputs per thread into the output tile, staged as
// four 32 x 32 boxes under the 128-byte swizzle in the staging buffer the
// vertical pass has consumed; one thread writes them with TMA stores clipped
// to the image.  Border tiles (whose windows are completed by the threads)
// are walked first (border_first_tile).
#include <algorithm>

#include "adjwt_internal.h"
#include "device_common.cuh"
#include "tma.cuh"

namespace adjwt {

constexpr int kTmaMaxRadius = 12;

namespace {

constexpr int kTH = 32;    // output rows per tile
constexpr int kTW = 128;   // output columns per tile
constexpr int kRB = 16;    // outputs per thread per pass
constexpr int kPT = 288;   // threads: 9 warps (vertical pass items), 8 of them in the horizontal pass

__host__ __device__ constexpr int up4(int v) { return (v + 3) / 4 * 4; }
__host__ __device__ constexpr int up32(int v) { return (v + 31) / 32 * 32; }

template <int R>
struct TG {
  static constexpr int XA = up4(R);           // staged columns left of the tile
  static constexpr int BW = kTW + 2 * XA;     // box width (floats)
  static constexpr int BH = kTH + 2 * R;      // box height (rows)
  static constexpr int BUF = up32(BH * BW);   // floats per staging buffer (128-byte multiple)
  static constexpr int VC = kTW + 2 * R;      // columns of the vertical-pass output
  static constexpr int TP = VC | 1;           // odd pitch of T
  // the output tile is staged as four 32 x 32 boxes (128-byte rows, 128-byte
  // swizzle) in the staging buffer the vertical pass has consumed, from a
  // 1024-byte boundary inside it
  static constexpr int OUT0 = 0;
  static constexpr int OUT1 = (BUF + 255) / 256 * 256;
  static_assert(kTH * kTW <= BUF && OUT1 + kTH * kTW <= 2 * BUF, "the staged output tile fits");
  static constexpr size_t smem_bytes() {
    return 1024 + (size_t)(2 * BUF + kTH * TP) * 4 + BH + BW;
  }
};

struct TmaBlurArgs {
  const float* in;
  const float* b;      // forward: subtract b (may be null)
  float* out;          // may be null (forward: residual norm only)
  double* partials;    // forward: per-CTA 1/2 sum (R u - b)^2 (may be null)
  int* status;         // device status word (timeouts)
  int rows, cols, pitch, bc;  // bc: 0 zero, 1 sym, 3 per
  int sym_taps;        // both tap vectors palindromic: R^* needs no orientation flips
  int ir0, ir1, ic0, ic1;  // tiles whose window stays inside the image (walked after the others)
  float pr[2 * kTmaMaxRadius + 1], pc[2 * kTmaMaxRadius + 1];  // taps as given, padded to 2R+1
};

__device__ __forceinline__ bool odd_period(int x, int N) { return (floor_div(x, N) & 1) != 0; }

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Source of virtual index x under the symmetric / periodic extension, with a
// division-free path for the first reflection or wrap.
__device__ __forceinline__ int ext_near(int x, int N, int mode) {
  if (x >= 0 && x < N) return x;
  if (x >= -N && x < 2 * N) {
    if (mode == 1) return x < 0 ? -1 - x : 2 * N - 1 - x;
    return x < 0 ? x + N : x - N;
  }
  return ext_src(x, N, mode);
}

// Off-image cells of a staged window, as strips: rows above / below the
// image (full width), then the columns left / right of it on the other rows.
// The TMA unit zero-fills them; under the symmetric and periodic extensions
// the threads overwrite them with their sources.
template <int R>
struct Strips {
  int x0, y0, rlo, rhi, clo, chi, side, ntop, nbot, total;
  __device__ __forceinline__ Strips(const TmaBlurArgs& a, int x0_, int y0_) : x0(x0_), y0(y0_) {
    using G = TG<R>;
    rlo = clampi(R - y0, 0, G::BH);
    rhi = clampi(a.rows - (y0 - R), rlo, G::BH);
    clo = clampi(G::XA - x0, 0, G::BW);
    chi = clampi(a.cols - (x0 - G::XA), clo, G::BW);
    side = clo + (G::BW - chi);
    ntop = rlo * G::BW;
    nbot = (G::BH - rhi) * G::BW;
    total = ntop + nbot + (rhi - rlo) * side;
  }
  // staged cell index of off-image cell i < total
  __device__ __forceinline__ int cell(int i) const {
    using G = TG<R>;
    if (i < ntop) return i;
    if (i < ntop + nbot) return rhi * G::BW + (i - ntop);
    const int j = i - ntop - nbot, rr = j / side, k = j - rr * side;
    return (rlo + rr) * G::BW + (k < clo ? k : chi + (k - clo));
  }
  __device__ __forceinline__ float load(const TmaBlurArgs& a, int mode, int c) const {
    using G = TG<R>;
    const int rr = c / G::BW, cc = c - rr * G::BW;
    const int sr = ext_near(y0 - R + rr, a.rows, mode), sc = ext_near(x0 - G::XA + cc, a.cols, mode);
    if (!in_bounds(a.status, sr >= 0 && sr < a.rows && sc >= 0 && sc < a.cols)) return 0.0f;
    return __ldg(a.in + (size_t)sr * a.pitch + sc);
  }
};

constexpr int kFillRegs = 6;  // off-image cells per thread fetched before the TMA wait

// T[r][c] = sum_t w[t] S[r + t][c + XA - R]; r < kTH, c < VC
template <int R, bool FLIP>
__device__ __forceinline__ void vertical(const float* __restrict__ S, float* __restrict__ T, const float (&w)[2 * R + 1],
                                         const unsigned char* __restrict__ flip_r) {
  using G = TG<R>;
  constexpr int K = 2 * R + 1, NW = kRB + 2 * R;
  for (int item = threadIdx.x; item < 2 * G::VC; item += kPT) {
    const int rb = item >= G::VC ? 1 : 0, c = item - rb * G::VC;
    const float* src = S + kRB * rb * G::BW + c + (G::XA - R);
    float acc[kRB];
#pragma unroll
    for (int o = 0; o < kRB; ++o) acc[o] = 0.0f;
#pragma unroll
    for (int j = 0; j < NW; ++j) {
      const float v = src[j * G::BW];
      bool f = false;
      if (FLIP) f = flip_r[kRB * rb + j] != 0;
#pragma unroll
      for (int o = 0; o < kRB; ++o) {
        const int t = j - o;
        if (t >= 0 && t < K) acc[o] = fmaf(FLIP ? (f ? w[K - 1 - t] : w[t]) : w[t], v, acc[o]);
      }
    }
    float* dst = T + kRB * rb * G::TP + c;
#pragma unroll
    for (int o = 0; o < kRB; ++o) dst[o * G::TP] = acc[o];
  }
}

// out[y0 + r][x0 + 16 blk + o] = sum_t w[t] T[r][16 blk + o + t] (- b), warp = blk, lane = r
template <int R, bool ADJ, bool FLIP>
__device__ __forceinline__ void horizontal(const float* __restrict__ T, const TmaBlurArgs& a, int x0, int y0,
                                           const float (&w)[2 * R + 1], const unsigned char* __restrict__ flip_c,
                                           float& sq, float* __restrict__ St) {
  using G = TG<R>;
  constexpr int K = 2 * R + 1, NW = kRB + 2 * R;
  const int warp = threadIdx.x >> 5, r = threadIdx.x & 31;
  if (warp >= kTW / kRB) return;
  const int y = y0 + r, x = x0 + kRB * warp;
  if (y >= a.rows || x >= a.cols) return;
  const bool full = x + kRB <= a.cols;
  float bv[kRB];
  const bool sub = !ADJ && a.b != nullptr;
  if (sub) {
    const float* bb = a.b + (size_t)y * a.pitch + x;
    if (full) {
#pragma unroll
      for (int q = 0; q < kRB / 4; ++q) {
        const float4 b4 = __ldg(reinterpret_cast<const float4*>(bb) + q);
        bv[4 * q] = b4.x;
        bv[4 * q + 1] = b4.y;
        bv[4 * q + 2] = b4.z;
        bv[4 * q + 3] = b4.w;
      }
    } else {
#pragma unroll
      for (int o = 0; o < kRB; ++o) bv[o] = x + o < a.cols ? __ldg(bb + o) : 0.0f;
    }
  }
  const float* src = T + r * G::TP + kRB * warp;
  float acc[kRB];
#pragma unroll
  for (int o = 0; o < kRB; ++o) acc[o] = 0.0f;
#pragma unroll
  for (int j = 0; j < NW; ++j) {
    const float v = src[j];
    bool f = false;
    if (FLIP) f = flip_c[kRB * warp + j] != 0;
#pragma unroll
    for (int o = 0; o < kRB; ++o) {
      const int t = j - o;
      if (t >= 0 && t < K) acc[o] = fmaf(FLIP ? (f ? w[K - 1 - t] : w[t]) : w[t], v, acc[o]);
    }
  }
  if (sub) {
#pragma unroll
    for (int o = 0; o < kRB; ++o) acc[o] -= bv[o];
  }
  if (!ADJ && a.partials) {
#pragma unroll
    for (int o = 0; o < kRB; ++o)
      if (full || x + o < a.cols) sq = fmaf(acc[o], acc[o], sq);
  }
  if (!a.out) return;
  // staged for the bulk stores (which write only the pixels inside the image):
  // 16-byte chunk c of row r of box x/32 at chunk position c xor (r mod 8), so
  // a quarter warp (8 consecutive rows, same chunk) hits 8 distinct bank groups
#pragma unroll
  for (int q = 0; q < kRB / 4; ++q) {
    const int col = kRB * warp + 4 * q;
    float* d = St + (col >> 5) * (kTH * 32) + r * 32 + ((((col >> 2) & 7) ^ (r & 7)) << 2);
    *reinterpret_cast<float4*>(d) = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
  }
}

// FLIPS: R^* of a symmetric image with taps that are not palindromic, the one
// case that needs the orientation-aware taps at border tiles; the other
// instantiations carry no code for them (a smaller loop body).
template <int R, bool ADJ, bool FLIPS>
__global__ void __launch_bounds__(kPT, (R <= 8 ? 3 : 2)) k_blur_tma(const __grid_constant__ CUtensorMap map,
                                                                           const __grid_constant__ CUtensorMap mo,
                                                                           const TmaBlurArgs a) {
  pdl_entry();
  using G = TG<R>;
  constexpr int K = 2 * R + 1;
  extern __shared__ unsigned char dyn[];
  __shared__ uint64_t bar[2];
  __shared__ double red[kPT / 32];
  float* buf0 = reinterpret_cast<float*>(dyn + ((1024 - (smem_u32(dyn) & 1023)) & 1023));  // buffer b at buf0 + b * BUF
  float* T = buf0 + 2 * G::BUF;
  unsigned char* flip_r = reinterpret_cast<unsigned char*>(T + kTH * G::TP);
  unsigned char* flip_c = flip_r + G::BH;

  const int tid = threadIdx.x;
  const int tiles_x = (a.cols + kTW - 1) / kTW;
  const int ntiles = tiles_x * ((a.rows + kTH - 1) / kTH);
  const int mode = a.bc == 3 ? 2 : a.bc;
  // taps: R is a convolution (reversed taps), R^* a correlation (taps as given)
  float wr[K], wc[K];
#pragma unroll
  for (int t = 0; t < K; ++t) {
    wr[t] = ADJ ? a.pr[t] : a.pr[K - 1 - t];
    wc[t] = ADJ ? a.pc[t] : a.pc[K - 1 - t];
  }
  // does the staged window leave the image?
  auto border = [&](int x0, int y0) {
    return y0 - R < 0 || x0 - G::XA < 0 || y0 + kTH + R > a.rows || x0 + kTW + G::XA > a.cols;
  };

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();

  uint32_t phase = 0, pending = 0;  // per buffer: parity of the next wait, copy in flight
  const int tiles_y = (a.rows + kTH - 1) / kTH;
  auto origin = [&](int t, int& y0, int& x0) {  // border tiles first (see border_first_tile)
    int ty, tx;
    border_first_tile(t, tiles_x, tiles_y, a.ir0, a.ir1, a.ic0, a.ic1, &ty, &tx);
    y0 = ty * kTH;
    x0 = tx * kTW;
  };
  auto issue = [&](int t, int b) {
    int y0, x0;
    origin(t, y0, x0);
    if (tid == 0) {
      fence_proxy_async();
      mbar_arrive_expect_tx(&bar[b], G::BH * G::BW * 4);
      tma_load_2d(buf0 + b * G::BUF, &map, &bar[b], x0 - G::XA, y0 - R);
    }
    pending |= 1u << b;
  };
  auto drain = [&]() {
    for (int b = 0; b < 2; ++b)
      if (pending & (1u << b)) mbar_wait(&bar[b], (phase >> b) & 1);
  };

  float sq = 0.0f;
  int t = blockIdx.x, b = 0;
  if (t < ntiles) issue(t, 0);
  for (; t < ntiles; t += gridDim.x, b ^= 1) {
    int y0, x0;
    origin(t, y0, x0);
    // off-image cells of a border window: fetch them while the copy is in flight
    const bool edge = border(x0, y0);
    const bool fill = edge && a.bc != 0;
    Strips<R> st(a, x0, y0);
    float fv[kFillRegs];
    if (fill) {
#pragma unroll
      for (int u = 0; u < kFillRegs; ++u) {
        const int i = tid + u * kPT;
        fv[u] = i < st.total ? st.load(a, mode, st.cell(i)) : 0.0f;
      }
    }
    bool ok = true;
    if (pending & (1u << b)) {
      ok = mbar_wait(&bar[b], (phase >> b) & 1);
      if (ok) {
        phase ^= 1u << b;
        pending &= ~(1u << b);
      }
    }
    if (!__syncthreads_and(ok)) {
      if (tid == 0) record_status(a.status, ADJWT_ERR_TIMEOUT);
      drain();
      if (tid == 0) bulk_wait_all();
      return;
    }
    float* S = buf0 + b * G::BUF;
    if (fill) {
#pragma unroll
      for (int u = 0; u < kFillRegs; ++u) {
        const int i = tid + u * kPT;
        if (i < st.total) S[st.cell(i)] = fv[u];
      }
      for (int i = tid + kFillRegs * kPT; i < st.total; i += kPT) {  // large overhangs (tiny images)
        const int c = st.cell(i);
        S[c] = st.load(a, mode, c);
      }
      __syncthreads();
    }
    // the vertical pass consumes this staging buffer; the other one (whose
    // staged output tile the previous tile's bulk stores have read) then
    // takes the next tile's copy
    auto next = [&]() {
      if (t + gridDim.x < ntiles) {
        if (tid == 0) bulk_wait_read();
        issue(t + gridDim.x, b ^ 1);
      }
    };
    float* St = buf0 + (b ? G::OUT1 : G::OUT0);
    const bool flip = FLIPS && edge;
    if constexpr (FLIPS) {
      if (flip) {
      for (int i = tid; i < G::BH; i += kPT) flip_r[i] = odd_period(y0 - R + i, a.rows);
      for (int i = tid; i < G::VC; i += kPT) flip_c[i] = odd_period(x0 - R + i, a.cols);
      __syncthreads();
      vertical<R, true>(S, T, wr, flip_r);
      __syncthreads();
      next();
      horizontal<R, ADJ, true>(T, a, x0, y0, wc, flip_c, sq, St);
      }
    }
    if (!flip) {
      vertical<R, false>(S, T, wr, nullptr);
      __syncthreads();
      next();
      horizontal<R, ADJ, false>(T, a, x0, y0, wc, nullptr, sq, St);
    }
    fence_proxy_async();  // the staged tile -> the bulk stores
    __syncthreads();      // also: T is rewritten next
    if (a.out && tid == 0) {
      // boxes wholly past the last column are skipped; the others are clipped to the image
#pragma unroll
      for (int bx = 0; bx < kTW / 32; ++bx)
        if (x0 + 32 * bx < a.cols) tma_store_2d(&mo, St + bx * (kTH * 32), x0 + 32 * bx, y0);
      bulk_commit();
    }
  }
  if (tid == 0) bulk_wait_all();  // the output is in global memory before the CTA exits
  if (!ADJ && a.partials) {
    const double tot = block_sum<kPT>((double)sq, red);
    if (tid == 0) a.partials[blockIdx.x] = 0.5 * tot;
  }
}

template <int R, bool ADJ, bool FLIPS = false>
int launch_r(const TmaBlurArgs& a, cudaStream_t s, int* nparts) {
  if (ADJ && !FLIPS && a.bc == 1 && !a.sym_taps) return launch_r<R, true, true>(a, s, nparts);
  using G = TG<R>;
  const size_t smem = G::smem_bytes();
  auto kern = k_blur_tma<R, ADJ, FLIPS>;
  ADJWT_CUDA_CHECK(set_smem(kern, smem));
  static int occ = 0;  // resident CTAs per SM (same on every device of one process)
  if (!occ) {
    int v = 0;
    ADJWT_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, kPT, smem));
    occ = std::max(v, 1);
  }
  const int ntiles = ((a.cols + kTW - 1) / kTW) * ((a.rows + kTH - 1) / kTH);
  const int grid = std::min(ntiles, sm_count() * occ);
  // interior tiles: windows inside the image (zero extension: no tile needs completing)
  TmaBlurArgs b = a;
  const int tx_n = (a.cols + kTW - 1) / kTW, ty_n = (a.rows + kTH - 1) / kTH;
  b.ir0 = b.ic0 = 0;
  b.ir1 = ty_n;
  b.ic1 = tx_n;
  if (a.bc != 0) {
    auto range = [](int n, int T, int lo_halo, int hi_halo, int N, int* lo, int* hi) {
      *lo = *hi = 0;
      bool found = false;
      for (int t = 0; t < n; ++t) {
        const bool in = t * T - lo_halo >= 0 && t * T + T + hi_halo <= N;
        if (in && !found) {
          *lo = t;
          found = true;
        }
        if (in) *hi = t + 1;
      }
    };
    range(ty_n, kTH, R, R, a.rows, &b.ir0, &b.ir1);
    range(tx_n, kTW, G::XA, G::XA, a.cols, &b.ic0, &b.ic1);
    if (b.ir1 <= b.ir0 || b.ic1 <= b.ic0) b.ir0 = b.ir1 = b.ic0 = b.ic1 = 0;
  }
  CUtensorMap map, mo;
  int rc = make_tmap_2d_f32(&map, a.in, a.rows, a.cols, a.pitch, G::BH, G::BW);
  if (rc) return rc;
  mo = map;
  if (a.out) {  // the output: 32 x 32 boxes, 128-byte swizzle, clipped to rows x cols
    rc = make_tmap_2d_f32_sw(&mo, a.out, a.rows, a.cols, a.pitch, kTH, 32, true);
    if (rc) return rc;
  }
  if (nparts) *nparts = grid;
  const char* name = ADJ ? "blur_adjoint" : (a.out ? "blur" : "blur_residual");
  ADJWT_TRACED(name, 0, s, pdl_launch(kern, grid, kPT, smem, s, map, mo, b));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  return ADJWT_OK;
}

}  // namespace

bool tma_blur_supported(const adjwt_blur_plan* p) {
  return (p->kr / 2) <= kTmaMaxRadius && (p->kc / 2) <= kTmaMaxRadius;
}

// The grid never exceeds the tile count, which bounds the partial slots.
int tma_blur_partial_slots(const adjwt_blur_plan* p) {
  return ((p->cols + kTW - 1) / kTW) * ((p->rows + kTH - 1) / kTH);
}

int launch_tma_blur(const adjwt_blur_plan* p, bool adjoint, const float* in, const float* b, float* out,
                    double* partials, cudaStream_t s, int* nparts) {
  const int R = std::max(p->kr / 2, p->kc / 2);
  TmaBlurArgs a{};
  a.in = in;
  a.b = adjoint ? nullptr : b;
  a.out = out;
  a.partials = adjoint ? nullptr : partials;
  a.status = device_status_ptr();
  a.rows = p->rows;
  a.cols = p->cols;
  a.pitch = p->image_pitch;
  a.bc = p->bc;
  a.sym_taps = 1;
  for (int t = 0; t < p->kr; ++t) a.sym_taps &= p->taps_r[t] == p->taps_r[p->kr - 1 - t];
  for (int t = 0; t < p->kc; ++t) a.sym_taps &= p->taps_c[t] == p->taps_c[p->kc - 1 - t];
  const int orr = R - p->kr / 2, oc = R - p->kc / 2;
  for (int t = 0; t < p->kr; ++t) a.pr[orr + t] = static_cast<float>(p->taps_r[t]);
  for (int t = 0; t < p->kc; ++t) a.pc[oc + t] = static_cast<float>(p->taps_c[t]);
  if (nparts) *nparts = 0;
  switch (R) {
#define ADJWT_R(r)                                                                       \
  case r:                                                                                \
    return adjoint ? launch_r<r, true>(a, s, nparts) : launch_r<r, false>(a, s, nparts);
    ADJWT_R(0) ADJWT_R(1) ADJWT_R(2) ADJWT_R(3) ADJWT_R(4) ADJWT_R(5) ADJWT_R(6)
    ADJWT_R(7) ADJWT_R(8) ADJWT_R(9) ADJWT_R(10) ADJWT_R(11) ADJWT_R(12)
#undef ADJWT_R
    default:
      return fail(ADJWT_ERR_INVALID_ARG, "TMA blur: radius above 12");
  }
}

}  // namespace adjwt
