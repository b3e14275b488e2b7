// Per-level choice of how a wavelet level runs, separately for W, for W^*
// (and W^dagger), and for W^* with the FISTA prox epilogue (a different
// kernel: it also reads and writes the iterate).  The candidates form a small
// grid over tile shape and pipeline: the tiled kernels alone (32 x 32 output
// tiles, one tile per CTA, no copy pipeline), or the persistent TMA-staged
// kernels (32 x 128 output tiles for W, 16 x 64 coefficient tiles for W^*,
// the next tile's copy in flight) with as many resident CTAs per SM as fit,
// or with one or two (more tiles per CTA go through its pipeline, fewer CTAs
// hide each other's latency).  The choice is measured: adjwt_wt_plan_autotune
// times whole transforms with each eligible level set to each candidate
// (greedy, level by level, the other levels at their current setting) and
// keeps the fastest (the default, the TMA kernel with as many CTAs as fit,
// unless another candidate wins by 3 %), then stores the result for the
// plan's size class (rows, cols, levels, wavelet, boundary, device), which
// every plan created later for that class applies.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "adjwt_internal.h"

namespace adjwt {
namespace {

using Key = std::tuple<int, int, int, int, int, int>;  // device, rows, cols, levels, wavelet, boundary
constexpr int kOps = 3;  // W, W^* / W^dagger, W^* with the prox epilogue
struct Choice {
  unsigned char off[kOps][kMaxLevels];
  unsigned char ctas[kOps][kMaxLevels];
};
std::mutex g_mu;
std::map<Key, Choice> g_cache;

bool key_of(const adjwt_wt_plan* p, Key* k) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  *k = Key{dev, p->rows, p->cols, p->levels, p->wavelet, p->bc};
  return true;
}

bool uses(const adjwt_wt_plan* p, int op, int j) {
  if (op != 0) return ana_tma_level(p, j, op == 2);
  int r0, r1, c0, c1;
  synth_tma_rect(p, j, &r0, &r1, &c0, &c1);
  return r1 > r0 && c1 > c0;
}

// Level j of operator op can take the TMA kernel under the size rule.
bool eligible(adjwt_wt_plan* p, int op, int j) {
  const unsigned char save = p->tma_off[op][j - 1];
  p->tma_off[op][j - 1] = 0;
  const bool e = uses(p, op, j);
  p->tma_off[op][j - 1] = save;
  return e;
}

struct DeviceBuffers {
  void* coeffs = nullptr;
  void* image = nullptr;
  void* ws = nullptr;
  void* y = nullptr;  // second iterate for the prox variant
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ~DeviceBuffers() {
    if (coeffs) cudaFree(coeffs);
    if (image) cudaFree(image);
    if (ws) cudaFree(ws);
    if (y) cudaFree(y);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

}  // namespace

void apply_tuning_cache(adjwt_wt_plan* p) {
  Key k;
  if (!key_of(p, &k)) return;
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_cache.find(k);
  if (it == g_cache.end()) return;
  for (int op = 0; op < kOps; ++op)
    for (int j = 0; j < kMaxLevels; ++j) {
      p->tma_off[op][j] = it->second.off[op][j];
      p->tma_ctas[op][j] = it->second.ctas[op][j];
    }
}

}  // namespace adjwt

using namespace adjwt;

extern "C" int adjwt_wt_plan_set_tma(adjwt_wt_plan* p, int op, int level, int enabled) {
  if (!p) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_wt_plan_set_tma: plan is NULL");
  if (op < 0 || op >= kOps) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_wt_plan_set_tma: op must be 0, 1 or 2");
  if (level < 1 || level > p->levels) return fail(ADJWT_ERR_SHAPE, "adjwt_wt_plan_set_tma: level out of range");
  p->tma_off[op][level - 1] = enabled ? 0 : 1;
  return ADJWT_OK;
}

extern "C" int adjwt_wt_plan_uses_tma(const adjwt_wt_plan* p, int op, int level, int* uses) {
  if (!p || !uses) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_wt_plan_uses_tma: NULL argument");
  if (op < 0 || op >= kOps) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_wt_plan_uses_tma: op must be 0, 1 or 2");
  if (level < 1 || level > p->levels) return fail(ADJWT_ERR_SHAPE, "adjwt_wt_plan_uses_tma: level out of range");
  *uses = adjwt::uses(p, op, level) ? 1 : 0;
  return ADJWT_OK;
}

extern "C" int adjwt_wt_plan_set_tma_ctas(adjwt_wt_plan* p, int op, int level, int ctas) {
  if (!p) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_wt_plan_set_tma_ctas: plan is NULL");
  if (op < 0 || op >= kOps) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_wt_plan_set_tma_ctas: op must be 0, 1 or 2");
  if (level < 1 || level > p->levels) return fail(ADJWT_ERR_SHAPE, "adjwt_wt_plan_set_tma_ctas: level out of range");
  if (ctas < 0 || ctas > 3) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_wt_plan_set_tma_ctas: ctas must be 0..3");
  p->tma_ctas[op][level - 1] = static_cast<unsigned char>(ctas);
  return ADJWT_OK;
}

extern "C" int adjwt_wt_plan_tma_ctas(const adjwt_wt_plan* p, int op, int level, int* ctas) {
  if (!p || !ctas) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_wt_plan_tma_ctas: NULL argument");
  if (op < 0 || op >= kOps) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_wt_plan_tma_ctas: op must be 0, 1 or 2");
  if (level < 1 || level > p->levels) return fail(ADJWT_ERR_SHAPE, "adjwt_wt_plan_tma_ctas: level out of range");
  *ctas = p->tma_ctas[op][level - 1];
  return ADJWT_OK;
}

extern "C" int adjwt_wt_plan_set_level_chain(adjwt_wt_plan* p, int enabled) {
  if (!p) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_wt_plan_set_level_chain: plan is NULL");
  p->chain_off = !enabled;
  return ADJWT_OK;
}

extern "C" int adjwt_wt_plan_chain_start(const adjwt_wt_plan* p, int op, int* first_level) {
  if (!p || !first_level) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_wt_plan_chain_start: NULL argument");
  if (op < 0 || op >= kOps) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_wt_plan_chain_start: op must be 0, 1 or 2");
  const int j0 = op == 0 ? syn_chain_start(p) : ana_chain_start(p, true, op == 2);
  *first_level = j0 <= p->levels ? j0 : 0;
  return ADJWT_OK;
}

extern "C" int adjwt_wt_plan_autotune(adjwt_wt_plan* p, int reps, int* from_cache, adjwt_stream_t stream) {
  if (!p) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_wt_plan_autotune: plan is NULL");
  if (reps < 1 || reps > 1000) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_wt_plan_autotune: reps must be in 1..1000");
  if (from_cache) *from_cache = 0;
  Key key;
  if (!key_of(p, &key)) return fail(ADJWT_ERR_CUDA, "adjwt_wt_plan_autotune: no current device");
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_cache.count(key)) {
      if (from_cache) *from_cache = 1;
    }
  }
  if (from_cache && *from_cache) {
    apply_tuning_cache(p);
    return ADJWT_OK;
  }
  DeviceBuffers d;
  const size_t cbytes = static_cast<size_t>(p->num_coeffs) * 4;
  const size_t ibytes = static_cast<size_t>(p->rows) * p->image_pitch * 4;
  const size_t wbytes = std::max<size_t>(adjwt_wt_workspace_size(p), 256);
  ADJWT_CUDA_CHECK(cudaMalloc(&d.coeffs, cbytes));
  ADJWT_CUDA_CHECK(cudaMalloc(&d.image, ibytes));
  ADJWT_CUDA_CHECK(cudaMalloc(&d.ws, wbytes));
  ADJWT_CUDA_CHECK(cudaMalloc(&d.y, cbytes));
  ADJWT_CUDA_CHECK(cudaMemsetAsync(d.y, 0, cbytes, stream));
  ADJWT_CUDA_CHECK(cudaMemsetAsync(d.coeffs, 0, cbytes, stream));
  ADJWT_CUDA_CHECK(cudaMemsetAsync(d.image, 0, ibytes, stream));
  ADJWT_CUDA_CHECK(cudaEventCreate(&d.e0));
  ADJWT_CUDA_CHECK(cudaEventCreate(&d.e1));
  auto* coeffs = static_cast<float*>(d.coeffs);
  auto* image = static_cast<float*>(d.image);
  // the LL ping-pong buffers of the workspace, split as the public entries do
  float* ll0 = static_cast<float*>(d.ws);
  float* ll1 = reinterpret_cast<float*>(static_cast<char*>(d.ws) + round_up(p->ll_buf_floats[0] * 4, 256));
  ProxArgs prox{};
  prox.x = coeffs;
  prox.y = static_cast<float*>(d.y);
  prox.step = 1.0f;
  prox.thresh = 1e-3f;
  prox.beta = 0.5f;

  // milliseconds of `reps` back-to-back calls after one untimed call
  auto time_op = [&](int op, float* ms) -> int {
    for (int i = 0; i <= reps; ++i) {
      if (i == 1) ADJWT_CUDA_CHECK(cudaEventRecord(d.e0, stream));
      int rc;
      if (op == 0)
        rc = wt_synth(p, coeffs, image, d.ws, wbytes, stream);
      else if (op == 1)
        rc = wt_synth_adjoint(p, image, coeffs, d.ws, wbytes, stream);
      else
        rc = launch_wt_analysis(p, image, nullptr, true, prox, ll0, ll1, stream, nullptr);
      if (rc) return rc;
    }
    ADJWT_CUDA_CHECK(cudaEventRecord(d.e1, stream));
    ADJWT_CUDA_CHECK(cudaEventSynchronize(d.e1));
    ADJWT_CUDA_CHECK(cudaEventElapsedTime(ms, d.e0, d.e1));
    return ADJWT_OK;
  };
  // candidates: (tiled only) and (TMA kernel, CTAs per SM: as many as fit, 1, 2)
  constexpr int kCand = 4;
  const unsigned char cand_off[kCand] = {0, 1, 0, 0}, cand_ctas[kCand] = {0, 0, 1, 2};
  for (int op = 0; op < kOps; ++op)
    for (int j = 1; j <= p->levels; ++j) {
      if (!eligible(p, op, j)) continue;
      float ms[kCand] = {};
      int rc = ADJWT_OK;
      for (int c = 0; c < kCand && !rc; ++c) {
        p->tma_off[op][j - 1] = cand_off[c];
        p->tma_ctas[op][j - 1] = cand_ctas[c];
        rc = time_op(op, &ms[c]);
      }
      int best = 0;  // the default must be beaten by 3 %: timing noise keeps it
      for (int c = 1; c < kCand && !rc; ++c)
        if (ms[c] < 0.97f * ms[0] && ms[c] < ms[best]) best = c;
      p->tma_off[op][j - 1] = rc ? 0 : cand_off[best];
      p->tma_ctas[op][j - 1] = rc ? 0 : cand_ctas[best];
      if (rc) return rc;
    }
  Choice c{};
  for (int op = 0; op < kOps; ++op)
    for (int j = 0; j < kMaxLevels; ++j) {
      c.off[op][j] = p->tma_off[op][j];
      c.ctas[op][j] = p->tma_ctas[op][j];
    }
  std::lock_guard<std::mutex> lock(g_mu);
  g_cache[key] = c;
  return ADJWT_OK;
}
