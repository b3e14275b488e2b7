// Plan construction: level sizes, packed band layout, extension weight tables.
//
// Level j (1-based) maps LL_{j-1} (N_r x N_c; LL_0 = image) to four bands of
// n_r x n_c.  For ZERO / SYM / PPD each axis is extended by L' = L - 1
// samples per side (Sec. I-A) and analysed by the full zero-padded transform,
// so n = floor((N + 3L')/2); for the critically sampled circular mode PER,
// n = N/2.  The adjoint needs (E^dagger)^* = E diag(1/c), c[i] = number of
// extended samples that copy input sample i (the 1/2 and 1/3 entries of the
// closed forms in Sec. I-A); those weights are tabulated per level and axis.
#include <algorithm>
#include <cmath>

#include "adjwt_internal.h"

namespace adjwt {
namespace {

int band_len(int N, int L, int bc) { return bc == kPer ? N / 2 : (N + 3 * (L - 1)) / 2; }

int ext_src(long x, long N, int bc) {
  if (bc == kZero) return (x >= 0 && x < N) ? static_cast<int>(x) : -1;
  if (bc == kSym) {
    long m = x % (2 * N);
    if (m < 0) m += 2 * N;
    return static_cast<int>(m < N ? m : 2 * N - 1 - m);
  }
  long m = x % N;
  if (m < 0) m += N;
  return static_cast<int>(m);
}

}  // namespace

std::vector<float> inverse_copy_counts(int N, int Lp, int bc) {
  std::vector<int> c(N, 0);
  for (long x = -Lp; x < N + Lp; ++x) {
    int s = ext_src(x, N, bc);
    if (s >= 0) c[s]++;
  }
  std::vector<float> w(N);
  for (int i = 0; i < N; ++i) w[i] = static_cast<float>(1.0 / c[i]);
  return w;
}

}  // namespace adjwt

using namespace adjwt;

extern "C" int adjwt_wt_plan_create(adjwt_wt_plan** out, int rows, int cols, int levels, int wavelet, int bc) {
  if (!out) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_wt_plan_create: out is NULL");
  *out = nullptr;
  if (bc < ADJWT_BC_ZERO || bc > ADJWT_BC_PER) return fail(ADJWT_ERR_INVALID_ARG, "unknown boundary mode");
  if (rows < 1 || cols < 1 || levels < 1 || levels > kMaxLevels)
    return fail(ADJWT_ERR_SHAPE, "need rows, cols >= 1 and 1 <= levels <= 16");
  if (rows > (1 << 24) || cols > (1 << 24)) return fail(ADJWT_ERR_SHAPE, "image side above 2^24");
  FilterBank fb;
  if (!make_filter_bank(wavelet, &fb)) return fail(ADJWT_ERR_INVALID_ARG, "unknown wavelet");
  if (bc == kPer && ((rows % (1 << levels)) || (cols % (1 << levels))))
    return fail(ADJWT_ERR_SHAPE, "PER needs rows and cols divisible by 2^levels");
  const int Lp = fb.L - 1;

  auto* p = new adjwt_wt_plan();
  p->rows = rows;
  p->cols = cols;
  p->levels = levels;
  p->wavelet = wavelet;
  p->bc = bc;
  p->fb = fb;
  p->image_pitch = static_cast<int>(round_up(cols, 4));
  p->lv.resize(levels);

  int Nr = rows, Nc = cols;
  std::vector<std::pair<int, int>> nsz(levels);
  for (int j = 1; j <= levels; ++j) {
    Level& L = p->lv[j - 1];
    const int nr = band_len(Nr, fb.L, bc), nc = band_len(Nc, fb.L, bc);
    L.ax[0] = {Nr, nr, 0, nullptr};
    L.ax[1] = {Nc, nc, 0, nullptr};
    L.in_pitch = (j == 1) ? p->image_pitch : static_cast<int>(round_up(Nc, 4));
    L.band_pitch = static_cast<int>(round_up(nc, 4));
    // The tiled reconstruction kernel folds at most one mirror copy per side and
    // stages at most kSynthTile + 2L' virtual rows per tile; sizes outside that
    // (N <= 2L', or, symmetric, a first tile that also holds the last L' rows
    // while N > kSynthTile) take the per-pixel gather kernel.
    auto needs_gather = [&](int N) {
      if (bc != kSym && bc != kPpd) return false;
      if (N <= 2 * Lp) return true;
      return bc == kSym && N > kSynthTile && N < kSynthTile + Lp;
    };
    L.generic_synth = needs_gather(Nr) || needs_gather(Nc);
    nsz[j - 1] = {nr, nc};
    Nr = nr;
    Nc = nc;
  }
  // packed order: LL_J, LH_J, HL_J, HH_J, LH_{J-1}, ...
  int64_t off = 0;
  auto add_band = [&](int j, int slot) {
    const Level& L = p->lv[j - 1];
    p->band_offsets.push_back(off);
    p->band_rows.push_back(L.ax[0].n);
    p->band_cols.push_back(L.ax[1].n);
    p->band_pitch.push_back(L.band_pitch);
    p->lv[j - 1].off_band[slot] = off;
    off += static_cast<int64_t>(L.ax[0].n) * L.band_pitch;
  };
  for (auto& L : p->lv)
    for (auto& o : L.off_band) o = -1;
  add_band(levels, 0);
  for (int j = levels; j >= 1; --j)
    for (int s = 1; s <= 3; ++s) add_band(j, s);
  p->num_coeffs = off;

  // LL ping-pong buffers: LL_j (j < J) lives in buffer j % 2
  p->ll_buf_floats[0] = p->ll_buf_floats[1] = 0;
  for (int j = 1; j < levels; ++j) {
    const Level& L = p->lv[j - 1];
    int64_t sz = static_cast<int64_t>(L.ax[0].n) * L.band_pitch;
    p->ll_buf_floats[j % 2] = std::max(p->ll_buf_floats[j % 2], sz);
  }
  // transforms of two or more levels may run a level chain, whose counters
  // sit past the LL data of the second buffer
  if (levels >= 2) p->ll_buf_floats[1] = round_up(p->ll_buf_floats[1], 64) + kChainCounterFloats;

  // 1/c tables for the weighted extension (E^dagger)^* and the fold E^dagger
  std::vector<float> host;
  std::vector<std::pair<int, int64_t>> where;  // (level*2+axis, offset)
  if (bc == kSym || bc == kPpd) {
    for (int j = 1; j <= levels; ++j)
      for (int a = 0; a < 2; ++a) {
        std::vector<float> w = inverse_copy_counts(p->lv[j - 1].ax[a].N, Lp, bc);
        where.push_back({(j - 1) * 2 + a, static_cast<int64_t>(host.size())});
        host.insert(host.end(), w.begin(), w.end());
        while (host.size() % 4) host.push_back(0.0f);
      }
  }
  if (!host.empty()) {
    cudaError_t e = cudaMalloc(&p->d_tables, host.size() * sizeof(float));
    if (e == cudaSuccess)
      e = cudaMemcpy(p->d_tables, host.data(), host.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      if (p->d_tables) cudaFree(p->d_tables);
      delete p;
      return cuda_fail(e, "adjwt_wt_plan_create: table upload");
    }
    for (auto& w : where) p->lv[w.first / 2].ax[w.first % 2].winv = p->d_tables + w.second;
  }
  apply_tuning_cache(p);
  *out = p;
  return ADJWT_OK;
}

extern "C" void adjwt_wt_plan_destroy(adjwt_wt_plan* p) {
  if (!p) return;
  if (p->d_tables) cudaFree(p->d_tables);
  delete p;
}

extern "C" int adjwt_wt_layout(const adjwt_wt_plan* p, int64_t* num_coeffs, int64_t* band_offsets, int* band_rows,
                               int* band_cols, int* band_pitch, int* image_pitch) {
  if (!p) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_wt_layout: plan is NULL");
  if (num_coeffs) *num_coeffs = p->num_coeffs;
  const size_t nb = p->band_offsets.size();
  for (size_t i = 0; i < nb; ++i) {
    if (band_offsets) band_offsets[i] = p->band_offsets[i];
    if (band_rows) band_rows[i] = p->band_rows[i];
    if (band_cols) band_cols[i] = p->band_cols[i];
    if (band_pitch) band_pitch[i] = p->band_pitch[i];
  }
  if (image_pitch) *image_pitch = p->image_pitch;
  return ADJWT_OK;
}

extern "C" size_t adjwt_wt_workspace_size(const adjwt_wt_plan* p) {
  if (!p) return 0;
  return static_cast<size_t>(round_up(p->ll_buf_floats[0] * 4, 256) + round_up(p->ll_buf_floats[1] * 4, 256)) + 256;
}

extern "C" int adjwt_wt_filters(const adjwt_wt_plan* p, double* dec_lo, double* dec_hi, double* rec_lo,
                                double* rec_hi, int* L) {
  if (!p) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_wt_filters: plan is NULL");
  for (int k = 0; k < p->fb.L; ++k) {
    if (dec_lo) dec_lo[k] = p->fb.dec_lo[k];
    if (dec_hi) dec_hi[k] = p->fb.dec_hi[k];
    if (rec_lo) rec_lo[k] = p->fb.rec_lo[k];
    if (rec_hi) rec_hi[k] = p->fb.rec_hi[k];
  }
  if (L) *L = p->fb.L;
  return ADJWT_OK;
}

// ------------------------------------------------------------------ blur plan
extern "C" int adjwt_blur_plan_create(adjwt_blur_plan** out, int rows, int cols, const double* taps_r, int kr,
                                      const double* taps_c, int kc, int bc) {
  if (!out) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_blur_plan_create: out is NULL");
  *out = nullptr;
  if (!taps_r || !taps_c) return fail(ADJWT_ERR_INVALID_ARG, "blur taps are NULL");
  if (bc != ADJWT_BC_ZERO && bc != ADJWT_BC_SYM && bc != ADJWT_BC_PER)
    return fail(ADJWT_ERR_INVALID_ARG, "blur boundary must be ZERO, SYM or PER");
  if (kr < 1 || kc < 1 || kr % 2 == 0 || kc % 2 == 0 || kr > 2 * kMaxBlurRadius + 1 ||
      kc > 2 * kMaxBlurRadius + 1)
    return fail(ADJWT_ERR_INVALID_ARG, "blur taps must have odd length <= 65");
  if (rows < 1 || cols < 1 || rows > (1 << 24) || cols > (1 << 24))
    return fail(ADJWT_ERR_SHAPE, "blur image must be at least 1 x 1");
  for (int i = 0; i < kr; ++i)
    if (!std::isfinite(taps_r[i])) return fail(ADJWT_ERR_INVALID_ARG, "non-finite blur tap");
  for (int i = 0; i < kc; ++i)
    if (!std::isfinite(taps_c[i])) return fail(ADJWT_ERR_INVALID_ARG, "non-finite blur tap");
  auto* p = new adjwt_blur_plan();
  p->rows = rows;
  p->cols = cols;
  p->bc = bc;
  p->kr = kr;
  p->kc = kc;
  p->image_pitch = static_cast<int>(round_up(cols, 4));
  for (int i = 0; i < kr; ++i) p->taps_r[i] = taps_r[i];
  for (int i = 0; i < kc; ++i) p->taps_c[i] = taps_c[i];
  *out = p;
  return ADJWT_OK;
}

extern "C" void adjwt_blur_plan_destroy(adjwt_blur_plan* p) { delete p; }

extern "C" int adjwt_blur_image_pitch(const adjwt_blur_plan* p) { return p ? p->image_pitch : 0; }

namespace adjwt {
size_t blur_partials_bytes(const adjwt_blur_plan* p) {
  return static_cast<size_t>(round_up(static_cast<int64_t>(blur_partial_slots(p)) * 8 + 8, 256));
}
}  // namespace adjwt

// partial sums, then one image-sized scratch buffer (R u - b between the two passes)
extern "C" size_t adjwt_blur_workspace_size(const adjwt_blur_plan* p) {
  if (!p) return 0;
  const size_t img = static_cast<size_t>(round_up(static_cast<int64_t>(p->rows) * p->image_pitch * 4, 256));
  return blur_partials_bytes(p) + img;
}
