// Multi-level 2D wavelet launches: W (reconstruction), W^* (exact adjoint,
// Eq. 4) and W^dagger (analysis).  Each level runs as its own launch of the
// tiled kernels below (whose per-tile bodies are in wt_tiles.cuh), of the
// persistent TMA kernels (wt_tma.cu) or both; the deepest tiled-only levels
// can instead run as one level-chain launch (opt-in).  The per-pixel gather
// kernel takes the periodic extension's far copies, tiny images (N <= 2L')
// and symmetric levels whose mirror copies straddle a tile boundary.
#include <algorithm>
#include <type_traits>

#include "adjwt_internal.h"
#include "device_common.cuh"
#include "tma.cuh"
#include "wt_tiles.cuh"

namespace adjwt {
namespace {

template <int L>
__global__ void __launch_bounds__(kAnaThreads, 2) k_analysis(const AnaArgs a) {
  pdl_entry();
  __shared__ AnaSmem<L> sm;
  __shared__ double red[kAnaThreads / 32];
  extern __shared__ float prox_slots[];  // kProxSlotBytes when the launch has prox bands, else none
  int tile_y, tile_x;
  border_tile(a.in_r0, a.in_r1, a.in_c0, a.in_c1, a.tiles_r, a.tiles_c, &tile_y, &tile_x);
  float l1 = 0.0f;
  analysis_tile<L, false>(a, tile_y, tile_x, l1, sm, prox_slots);
  if (a.l1) {
    const double tot = block_sum<kAnaThreads>((double)l1, red);
    if (threadIdx.x == 0) a.l1[blockIdx.y * gridDim.x + blockIdx.x] = tot;
  }
}

template <int L>
__global__ void __launch_bounds__(kThreads) k_synthesis(const SynArgs a) {
  pdl_entry();
  __shared__ SynSmem<L> sm;
  int tile_y, tile_x;
  border_tile(a.in_r0, a.in_r1, a.in_c0, a.in_c1, a.tiles_r, a.tiles_c, &tile_y, &tile_x);
  synthesis_tile<L, false>(a, tile_y, tile_x, sm);
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
  synthesis_gather_pixel<L, false>(a, tr, tc);
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
// (block barrier, then a release add by the counting thread, cumulative over
// the barrier).
__device__ __forceinline__ void chain_done(int* counters, int lev) {
  __syncthreads();
  if (threadIdx.x == 0) asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(counters + kChainDone + lev) : "memory");
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
  __shared__ AnaSmem<L> sm;
  __shared__ int s_word[2];
  __shared__ double red[kAnaThreads / 32];
  extern __shared__ float prox_slots[];
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
    analysis_tile<L, true>(s_a, ty, local - ty * s_a.tiles_c, l1_tile, sm, prox_slots);
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
  __shared__ SynSmem<L> sm;
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
    synthesis_tile<L, true>(s_a, ty, local - ty * s_a.tiles_c, sm);
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
  a.status = device_status_ptr();
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
    a.status = device_status_ptr();
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
