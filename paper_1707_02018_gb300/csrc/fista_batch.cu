// Batched FISTA engine: many independent deblurring problems (Eq. 1, each
// with its own image size, wavelet, depth and PSF) run `iters` FISTA
// iterations in ONE persistent launch.
//
// Work items.  One iteration of problem p is a chain of stages
//     MOM, W level J, ..., W level 1, R^*(R u - b), W^* level 1 (+prox), ..., W^* level J (+prox)
// (MOM advances the device-resident momentum t_k, beta_k).  A stage is cut
// into tiles: the tiled level bodies of wt_tiles.cuh (32 x 32 outputs) and
// the blur bodies (32 x 64 TMA windows, blur_window_tile.cuh, or gathered
// 64 x 64 tiles, blur_tile.cuh).  An item is one tile, or two to four
// consecutive tiles of a stage with many (tiles_per_item).  The
// items of an iteration are numbered stage-major across problems (stage
// slot s of every problem before slot s + 1 of any), iteration after
// iteration; CTAs take the next item number from a counter.
//
// Dependencies.  A stage may start once every tile of the previous stage of
// the same problem is done (the first stage: the last stage of the previous
// iteration).  Per-stage done counters grow monotonically over the launch, so
// the target of a wait is (iteration + 1) x (tiles of the stage waited on).
// A CTA only waits on items numbered below its own, all handed out to
// running CTAs, so the launch needs no co-residency.  Many problems keep
// other items ready while one problem waits.
//
// Waits are bounded (kWaitCycles, about a second): a CTA that gives up
// records ADJWT_ERR_TIMEOUT in the device status word and raises the
// launch's abort flag, on which every other CTA stops taking items and every
// wait returns.
//
// The objective F(x_k) = 1/2 ||R W x_k - b||^2 + lambda ||x_k||_1 runs as a
// second persistent launch over all problems (W on x_k, the blur residual
// norm, |x_k|, then a fixed-order sum per problem).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "adjwt_internal.h"
#include "blur_tile.cuh"
#include "blur_window_tile.cuh"
#include "device_common.cuh"
#include "tma.cuh"
#include "wt_tiles.cuh"

namespace adjwt {
namespace {

constexpr int kEngineThreads = 256;
constexpr int kEngineMaxRadius = 12;

// kBlur: the fused 64 x 64 blur tile (gathered windows); kBlurW: the 32 x 64
// tile from TMA-staged windows (problems whose R^* needs no orientation-aware
// taps: every boundary but the symmetric one with non-palindromic taps)
enum StageKind : int { kMom = 0, kSyn = 1, kBlur = 2, kAna = 3, kSum = 4, kL1 = 5, kGat = 6, kBlurW = 7 };
constexpr int kGatherPixels = kEngineThreads;  // pixels per item of a per-pixel gather level

// One stage of one problem's iteration.
struct Stage {
  int kind;
  int param;       // filter length L (kSyn, kAna, kL1) or padded blur radius (kBlur, kBlurW)
  int problem;
  int args;        // index into the argument array of its kind
  int ntiles, tiles_c;
  int prev;        // stage waited on (-1: none)
  int prev_items;  // its items
  int group;       // tiles per item (set when the stages are ordered)
  int prev_lag;    // 1: prev belongs to the previous iteration
  int part;        // first partial slot of its tiles (kBlur, kBlurW, kAna with prox, kL1), else -1
};

// Arguments of a kBlurW stage: the tensor maps over u and b (boxes of
// WG<R>) live in device memory next to the tile arguments.
struct BlurWinArgs {  // aligned as its tensor maps
  CUtensorMap umap, bmap;
  TiledArgs a;
};

struct ProbDev {
  double* mom;      // m[0] = t_k, m[1] = beta_k
  double* parts;    // partial slots: blur tiles first, then the |x| tiles
  int nblur, nl1;
  double lambda;
};

// Per item of one iteration: its stage's record and its tile, so that taking
// an item costs one dependent load (made while the previous item runs).
struct __align__(16) Item {
  int kind, param, problem, args, tiles_c, part;  // its stage's (Stage)
  int st;    // its stage
  int tile;  // its first tile within the stage
  int prev;  // the stage it waits on (-1: none)
  int pt2;   // that stage's items * 2, + 1 if it belongs to the previous iteration
  int ntl;   // its tiles (consecutive)
  int pad;
};

struct EngineArgs {
  const Item* items;       // per item of one iteration
  int items_per_iter;
  int iters;
  const SynArgs* syn;
  const AnaArgs* ana;
  const TiledArgs* blur;
  const BlurWinArgs* blurw;
  const ProbDev* prob;
  double* objectives;      // objective launch: one per problem
  int* counters;           // [0] next item, [1] abort flag, [2 + stage] tiles done
  int* status;
  int stall;               // wait self-test: the first item waits for a stage that never runs
};

constexpr int kCtrDone = 2;

// Bounded wait with acquire semantics until *ctr >= target, or the abort flag.
__device__ __forceinline__ bool engine_wait(const int* ctr, int target, const int* abort_flag) {
  const long long t0 = clock64();
  for (;;) {
    int v, ab;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
    if (v >= target) return true;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(ab) : "l"(abort_flag) : "memory");
    if (ab) return false;
    if (clock64() - t0 > kWaitCycles) return false;
    __nanosleep(64);
  }
}

// Argument block into shared memory by warps 1 .. 6 (meanwhile thread 0 is
// in the item's dependency wait and warp 7 publishes the previous item).
template <typename T>
__device__ __forceinline__ void copy_block_args(T* dst, const T* src) {
  static_assert(sizeof(T) % 4 == 0, "argument blocks are whole words");
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(dst);
  const int i0 = static_cast<int>(threadIdx.x) - 32;
  if (i0 >= 0 && i0 < kEngineThreads - 64)
    for (int i = i0; i < (int)(sizeof(T) / 4); i += kEngineThreads - 64) d[i] = s[i];
}

template <typename Fn>
__device__ __forceinline__ void with_L(int L, Fn&& fn) {
  switch (L) {
    case 2: fn(std::integral_constant<int, 2>()); break;
    case 4: fn(std::integral_constant<int, 4>()); break;
    case 8: fn(std::integral_constant<int, 8>()); break;
    default: fn(std::integral_constant<int, 10>()); break;
  }
}

// blur radius of the fused tile: exact from 2 to 9 (the radii of Gaussian
// PSFs with sigma up to 3), radii 0 and 1 padded to 2 and 10..12 to 12 (zero
// taps leave the operator unchanged)
__host__ __device__ constexpr int padded_radius(int r) { return r <= 2 ? 2 : r <= 9 ? r : 12; }

template <typename Fn>
__device__ __forceinline__ void with_R(int R, Fn&& fn) {
  switch (R) {
    case 2: fn(std::integral_constant<int, 2>()); break;
    case 3: fn(std::integral_constant<int, 3>()); break;
    case 4: fn(std::integral_constant<int, 4>()); break;
    case 5: fn(std::integral_constant<int, 5>()); break;
    case 6: fn(std::integral_constant<int, 6>()); break;
    case 7: fn(std::integral_constant<int, 7>()); break;
    case 8: fn(std::integral_constant<int, 8>()); break;
    case 9: fn(std::integral_constant<int, 9>()); break;
    default: fn(std::integral_constant<int, 12>()); break;
  }
}

union StageArgs {
  SynArgs syn;
  AnaArgs ana;
  TiledArgs blur;
};

constexpr int kL1Chunk = 8192;  // coefficients per |x| tile of the objective launch

struct L1Args {
  const float* x;
  int64_t n;
};

// Shared memory of the engine: the bodies' smem (one at a time) at the start,
// the prox slots of the analysis body after the largest analysis smem.
constexpr size_t kProxOffset = (sizeof(AnaSmem<10>) + 127) / 128 * 128;

// One body per call, kept out of line so that each is register-allocated on
// its own rather than all of them together in the engine loop.
template <int L>
__device__ __noinline__ void engine_syn(const SynArgs& a, int ty, int tx, unsigned char* dyn) {
  synthesis_tile<L, true>(a, ty, tx, *reinterpret_cast<SynSmem<L>*>(dyn));
}

template <int L>
__device__ __noinline__ void engine_gat(const SynArgs& a, int tr, int tc) {
  synthesis_gather_pixel<L, true>(a, tr, tc);
}

template <int L>
__device__ __noinline__ float engine_ana(const AnaArgs& a, int ty, int tx, unsigned char* dyn) {
  float l1 = 0.0f;
  analysis_tile<L, true, kEngineThreads>(a, ty, tx, l1, *reinterpret_cast<AnaSmem<L>*>(dyn),
                                         reinterpret_cast<float*>(dyn + kProxOffset));
  return l1;
}

template <int R>
__device__ __noinline__ float engine_blur_window(const TiledArgs& a, const CUtensorMap* umap, const CUtensorMap* bmap,
                                                 int ty, int tx, unsigned char* dyn) {
  return blur_window_tile<R>(a, umap, bmap, ty, tx, dyn);
}

template <int R>
__device__ __noinline__ float engine_blur(const TiledArgs& a, int ty, int tx, unsigned char* dyn, int* s_border) {
  float sq = 0.0f;
  blur_normal_tile<R, true>(a, ty, tx, reinterpret_cast<float*>(dyn), s_border, sq);
  return sq;
}

__global__ void __launch_bounds__(kEngineThreads, 3) k_fista_engine(const EngineArgs e, const L1Args* l1args) {
  pdl_entry();
  extern __shared__ __align__(128) unsigned char dyn[];
  __shared__ StageArgs s_args;
  __shared__ int s_word[2];  // [0] the item to run, [1] whether it may run
  __shared__ Item s_item;
  __shared__ double red[kEngineThreads / 32];
  __shared__ int s_border;
  const int tid = threadIdx.x;
  int* abort_flag = e.counters + 1;
  const int total = e.items_per_iter * e.iters;
  // Thread 0 holds two tickets ahead and loads the next item's record while
  // the current one runs, so that an item starts after one round trip: its
  // dependency wait, beside the copy of its argument block.  The smallest
  // unfinished ticket is still always some CTA's current item, whose
  // dependencies all have smaller tickets, so the launch makes progress.
  int n1 = 0, n2 = 0;
  Item nxt{};
  if (tid == 0) {
    const int t0 = atomicAdd(&e.counters[0], 1);
    n1 = atomicAdd(&e.counters[0], 1);
    if (t0 < total) s_item = e.items[t0 % e.items_per_iter];
    s_word[0] = t0;
  }
  __syncthreads();
  int cur_st = -1;  // stage whose argument block is in s_args
  for (;;) {
    const int item = s_word[0];
    if (item >= total) break;
    const Item I = s_item;
    const int st = I.st;
    if (tid == 0) {
      if (n1 < total) nxt = e.items[n1 % e.items_per_iter];
      n2 = atomicAdd(&e.counters[0], 1);
      const int it = item / e.items_per_iter, pt = I.pt2 >> 1;
      int target = (it + 1 - (I.pt2 & 1)) * pt;
      if (e.stall && item == 0) target = pt;  // a previous iteration that never ran
      // the abort flag and the first poll of the dependency are in flight together
      int ab;
      asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(ab) : "l"(abort_flag) : "memory");
      int go = 1;
      if (I.prev >= 0 && target > 0 && !engine_wait(&e.counters[kCtrDone + I.prev], target, abort_flag)) {
        record_status(e.status, ADJWT_ERR_TIMEOUT);
        atomicExch(abort_flag, 1);
        go = 0;
      }
      if (ab) go = 0;
      s_word[1] = go;
    }
    if (st != cur_st) {
      switch (I.kind) {
        case kSyn:
        case kGat:
          copy_block_args(&s_args.syn, &e.syn[I.args]);
          break;
        case kAna:
          copy_block_args(&s_args.ana, &e.ana[I.args]);
          break;
        case kBlur:
          copy_block_args(&s_args.blur, &e.blur[I.args]);
          break;
        case kBlurW:
          copy_block_args(&s_args.blur, &e.blurw[I.args].a);
          break;
        default:
          break;
      }
    }
    __syncthreads();
    if (!s_word[1]) break;
    for (int q = 0; q < I.ntl; ++q) {
      if (q > 0) __syncthreads();  // the previous tile is done with shared memory
      const int tile = I.tile + q;
      const int ty = tile / I.tiles_c, tx = tile - ty * I.tiles_c;
      switch (I.kind) {
        case kMom:
          if (tid == 0) {
            // device-resident momentum (the method cited in Sec. I-B):
            // t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2, beta_k = (t_k - 1) / t_{k+1}
            double* m = e.prob[I.problem].mom;
            const double t = __ldcg(m);
            const double t1 = 0.5 * (1.0 + sqrt(__dadd_rn(1.0, __dmul_rn(4.0 * t, t))));
            m[1] = (t - 1.0) / t1;
            m[0] = t1;
          }
          break;
        case kSyn:
          with_L(I.param, [&](auto Lc) { engine_syn<decltype(Lc)::value>(s_args.syn, ty, tx, dyn); });
          break;
        case kGat: {
          const int64_t idx = (int64_t)tile * kGatherPixels + tid;
          if (idx < (int64_t)s_args.syn.Nr * s_args.syn.Nc) {
            const int tr = static_cast<int>(idx / s_args.syn.Nc);
            const int tc = static_cast<int>(idx - (int64_t)tr * s_args.syn.Nc);
            with_L(I.param, [&](auto Lc) { engine_gat<decltype(Lc)::value>(s_args.syn, tr, tc); });
          }
          break;
        }
        case kAna: {
          float l1 = 0.0f;
          with_L(I.param, [&](auto Lc) { l1 = engine_ana<decltype(Lc)::value>(s_args.ana, ty, tx, dyn); });
          if (I.part >= 0) {
            const double tot = block_sum<kEngineThreads>((double)l1, red);
            if (tid == 0) e.prob[I.problem].parts[I.part + tile] = tot;
          }
          break;
        }
        case kBlur: {
          float sq = 0.0f;
          with_R(I.param, [&](auto Rc) { sq = engine_blur<decltype(Rc)::value>(s_args.blur, ty, tx, dyn, &s_border); });
          if (I.part >= 0) {
            const double tot = block_sum<kEngineThreads>((double)sq, red);
            if (tid == 0) e.prob[I.problem].parts[I.part + tile] = 0.5 * tot;
          }
          break;
        }
        case kBlurW: {
          const BlurWinArgs* w = &e.blurw[I.args];
          float sq = 0.0f;
          with_R(I.param, [&](auto Rc) {
            sq = engine_blur_window<decltype(Rc)::value>(s_args.blur, &w->umap, &w->bmap, ty, tx, dyn);
          });
          if (I.part >= 0) {
            const double tot = block_sum<kEngineThreads>((double)sq, red);
            if (tid == 0) e.prob[I.problem].parts[I.part + tile] = 0.5 * tot;
          }
          break;
        }
        case kL1: {
          const L1Args la = l1args[I.args];
          const int64_t i0 = (int64_t)tile * kL1Chunk;
          float acc = 0.0f;
          for (int64_t i = i0 + tid; i < la.n && i < i0 + kL1Chunk; i += kEngineThreads) acc += fabsf(__ldcg(la.x + i));
          const double tot = block_sum<kEngineThreads>((double)acc, red);
          if (tid == 0) e.prob[I.problem].parts[I.part + tile] = tot;
          break;
        }
        case kSum:
          if (tid == 0) {
            // F(x) = 1/2 ||R W x - b||^2 + lambda ||x||_1, partials added in a fixed order
            const ProbDev pd = e.prob[I.problem];
            double r = 0.0, l1 = 0.0;
            for (int i = 0; i < pd.nblur; ++i) r += __ldcg(pd.parts + i);
            for (int i = 0; i < pd.nl1; ++i) l1 += __ldcg(pd.parts + pd.nblur + i);
            e.objectives[I.problem] = r + pd.lambda * l1;
          }
          break;
        default:
          break;
      }
    }
    cur_st = st;
    if (tid == 0) {
      s_word[0] = n1;
      s_item = nxt;
      n1 = n2;
    }
    // every write of the tile happens before its count is published: block
    // barrier, then a release add by one thread (cumulative over the
    // barrier).  The first thread of warp 7 makes it, so that its fence runs
    // beside thread 0's work on the next item.
    __syncthreads();
    if (tid == kEngineThreads - 32)
      asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(e.counters + kCtrDone + st) : "memory");
  }
}

__global__ void k_batch_reset(double* const* mom, int count, double t) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) {
    mom[i][0] = t;
    mom[i][1] = 0.0;
  }
}

}  // namespace
}  // namespace adjwt

// ===================================================================== host
namespace adjwt {
namespace {

// Workspace of one problem: u and g images, the LL ping-pong buffers, the
// momentum (2 doubles) and the objective partials.
struct ProbWs {
  size_t u, g, ll0, ll1, mom, parts, bytes;
  int nblur, nl1;
};

// Whether a problem's blur stage takes the TMA-window tile: not under the
// symmetric boundary with non-palindromic taps (R^* would need
// orientation-aware taps at the border).
bool blur_window_ok(const adjwt_blur_plan* b) {
  if (b->bc != kSym) return true;
  for (int t = 0; t < b->kr; ++t)
    if (b->taps_r[t] != b->taps_r[b->kr - 1 - t]) return false;
  for (int t = 0; t < b->kc; ++t)
    if (b->taps_c[t] != b->taps_c[b->kc - 1 - t]) return false;
  return true;
}
int blur_tiles_c(const adjwt_blur_plan* b) { return blur_window_ok(b) ? (b->cols + kWW - 1) / kWW : (b->cols + kT - 1) / kT; }
int blur_tiles(const adjwt_blur_plan* b) {
  const int th = blur_window_ok(b) ? kWH : kT;
  return blur_tiles_c(b) * ((b->rows + th - 1) / th);
}
int l1_tiles(const adjwt_wt_plan* w) { return static_cast<int>((w->num_coeffs + kL1Chunk - 1) / kL1Chunk); }

ProbWs prob_ws(const adjwt_fista_problem& pr) {
  ProbWs w{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += static_cast<size_t>(round_up(static_cast<int64_t>(bytes), 256));
    return o;
  };
  const size_t img = (size_t)pr.wt->rows * pr.wt->image_pitch * sizeof(float);
  w.u = take(img);
  w.g = take(img);
  w.ll0 = take(std::max<int64_t>(pr.wt->ll_buf_floats[0], 1) * sizeof(float));
  w.ll1 = take(std::max<int64_t>(pr.wt->ll_buf_floats[1], 1) * sizeof(float));
  w.mom = take(2 * sizeof(double));
  w.nblur = blur_tiles(pr.blur);
  w.nl1 = l1_tiles(pr.wt);
  w.parts = take((size_t)(w.nblur + w.nl1) * sizeof(double));
  w.bytes = off;
  return w;
}

int blur_radius(const adjwt_blur_plan* b) { return padded_radius(std::max(b->kr / 2, b->kc / 2)); }

int check_batch_problem(const adjwt_fista_problem& pr, int i) {
  const std::string who = "fista_batch: problem " + std::to_string(i);
  if (!pr.wt || !pr.blur || !pr.b) return fail(ADJWT_ERR_INVALID_ARG, who + ": plan or b is NULL");
  if (pr.wt->rows != pr.blur->rows || pr.wt->cols != pr.blur->cols)
    return fail(ADJWT_ERR_SHAPE, who + ": wavelet and blur plans describe different images");
  if (pr.wt->bc == kPpd) return fail(ADJWT_ERR_SHAPE, who + ": the redundant periodic reconstruction is not batched");
  if (std::max(pr.blur->kr, pr.blur->kc) / 2 > kEngineMaxRadius)
    return fail(ADJWT_ERR_SHAPE, who + ": PSF radius above 12");
  if (!(pr.lambda >= 0.0) || !std::isfinite(pr.lambda)) return fail(ADJWT_ERR_INVALID_ARG, who + ": bad lambda");
  if (!(pr.lipschitz > 0.0) || !std::isfinite(pr.lipschitz))
    return fail(ADJWT_ERR_INVALID_ARG, who + ": lipschitz must be finite and > 0");
  if (pr.gradient != ADJWT_GRAD_ADJOINT && pr.gradient != ADJWT_GRAD_PINV)
    return fail(ADJWT_ERR_INVALID_ARG, who + ": unknown gradient mode");
  if ((reinterpret_cast<uintptr_t>(pr.b) & 15u) != 0) return fail(ADJWT_ERR_ALIGN, who + ": b not 16-byte aligned");
  return ADJWT_OK;
}

SynArgs syn_level(const adjwt_wt_plan* w, int j, const float* coeffs, float* out_image, float* const ll[2]) {
  const Level& L = w->lv[j - 1];
  SynArgs a{};
  for (int b = 0; b < 4; ++b) a.band[b] = (b == 0 && j < w->levels) ? ll[j % 2] : coeffs + L.off_band[b];
  a.band_pitch = L.band_pitch;
  a.out = (j == 1) ? out_image : ll[(j - 1) % 2];
  a.out_pitch = L.in_pitch;
  a.Nr = L.ax[0].N;
  a.Nc = L.ax[1].N;
  a.nr = L.ax[0].n;
  a.nc = L.ax[1].n;
  a.mode = w->bc;
  a.winv_r = L.ax[0].winv;
  a.winv_c = L.ax[1].winv;
  a.status = device_status_ptr();
  for (int t = 0; t < w->fb.L; ++t) {
    a.g[0][t] = static_cast<float>(w->fb.rec_lo[t]);
    a.g[1][t] = static_cast<float>(w->fb.rec_hi[t]);
  }
  a.tiles_c = (a.Nc + kTile - 1) / kTile;
  a.tiles_r = (a.Nr + kTile - 1) / kTile;
  return a;
}

AnaArgs ana_level(const adjwt_fista_problem& pr, int j, const float* in_image, float* x, float* y, float* const ll[2],
                  const double* beta_dev) {
  const adjwt_wt_plan* w = pr.wt;
  const Level& L = w->lv[j - 1];
  const bool adjoint = pr.gradient == ADJWT_GRAD_ADJOINT;
  AnaArgs a{};
  a.in = (j == 1) ? in_image : ll[(j - 1) % 2];
  a.in_pitch = L.in_pitch;
  a.Nr = L.ax[0].N;
  a.Nc = L.ax[1].N;
  a.nr = L.ax[0].n;
  a.nc = L.ax[1].n;
  a.mode = w->bc;
  a.winv_r = adjoint ? L.ax[0].winv : nullptr;
  a.winv_c = adjoint ? L.ax[1].winv : nullptr;
  a.out_pitch = L.band_pitch;
  a.status = device_status_ptr();
  for (int b = 0; b < 4; ++b) {
    if (b > 0 || j == w->levels) {
      a.px[b] = x + L.off_band[b];
      a.py[b] = y + L.off_band[b];
    } else {
      a.dst[b] = ll[j % 2];
    }
  }
  a.step = static_cast<float>(1.0 / pr.lipschitz);
  a.thresh = static_cast<float>(pr.lambda / pr.lipschitz);
  a.beta_dev = beta_dev;
  const FilterBank& fb = w->fb;
  for (int t = 0; t < fb.L; ++t) {
    if (adjoint) {  // dual analysis filters: synthesis filters reversed (Eq. 3, Eq. 4)
      a.flo[t] = static_cast<float>(fb.rec_lo[fb.L - 1 - t]);
      a.fhi[t] = static_cast<float>(fb.rec_hi[fb.L - 1 - t]);
    } else {
      a.flo[t] = static_cast<float>(fb.dec_lo[t]);
      a.fhi[t] = static_cast<float>(fb.dec_hi[t]);
    }
  }
  a.tiles_c = (L.band_pitch + kTile - 1) / kTile;
  a.tiles_r = (L.ax[0].n + kTile - 1) / kTile;
  return a;
}

// kBlurW arguments: the tile arguments and the tensor maps over u and b.
int window_args(const adjwt_fista_problem& pr, const float* u, float* g, double* partials, BlurWinArgs* out);

TiledArgs blur_args(const adjwt_fista_problem& pr, const float* u, float* g, double* partials) {
  const adjwt_blur_plan* p = pr.blur;
  const int R = blur_radius(p);
  TiledArgs a{};
  a.in = u;
  a.b = pr.b;
  a.out = g;
  a.partials = partials;
  a.rows = p->rows;
  a.cols = p->cols;
  a.pitch = p->image_pitch;
  a.bc = p->bc;
  a.status = device_status_ptr();
  const int orr = R - p->kr / 2, oc = R - p->kc / 2;
  for (int t = 0; t < p->kr; ++t) a.pr[orr + t] = static_cast<float>(p->taps_r[t]);
  for (int t = 0; t < p->kc; ++t) a.pc[oc + t] = static_cast<float>(p->taps_c[t]);
  return a;
}

}  // namespace
}  // namespace adjwt

namespace adjwt {
namespace {
// One launch's tables (the iteration launch and the objective launch).
struct BatchLaunch {
  EngineArgs args{};
  int nstages = 0;
  int items = 0;  // per iteration
};
}  // namespace
}  // namespace adjwt

struct adjwt_fista_batch {
  int count = 0;
  std::vector<adjwt_fista_problem> probs;
  std::vector<size_t> ws_off;
  void* dev = nullptr;            // tables, argument blocks, counters (owned)
  adjwt::BatchLaunch run, obj;
  const adjwt::L1Args* l1args = nullptr;
  double* const* mom_ptrs = nullptr;
  int* counters = nullptr;
  size_t counter_bytes = 0;
  size_t dyn = 0;
  int per_sm = 1;
  ~adjwt_fista_batch() {
    if (dev) cudaFree(dev);
  }
};

namespace adjwt {
namespace {

struct StageList {
  std::vector<Stage> st;  // in stage order, prev = index within the same problem's list (-1: none)
};

// Tiles per item: when the batch has far more tiles than the launch has CTAs,
// a stage with many tiles hands them out several at a time (consecutive
// tiles, one item), so that the per-item costs (ticket, dependency wait,
// argument copy, publishing) are shared.  A stage keeps one tile per item
// when it has fewer than 2 x kMinItems tiles, or when its stage slot across
// the batch holds fewer than 2 x kWaves tiles per CTA: few problems leave
// the CTAs short of items, and a coarser stage would only lengthen each
// problem's chain of dependent stages.
constexpr int kMinItems = 64;
constexpr int kWaves = 8;
int tiles_per_item(const Stage& S, int64_t slot_tiles, int ctas) {
  const int gmax = S.kind == kSyn ? 4 : (S.kind == kMom || S.kind == kSum) ? 1 : 2;
  const int64_t by_slot = slot_tiles / ((int64_t)kWaves * std::max(ctas, 1));
  return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>({gmax, S.ntiles / kMinItems, by_slot})));
}
int stage_items(const Stage& S) { return (S.ntiles + S.group - 1) / S.group; }

// Stage-major order across problems; prev indices become global; the first
// stage of a problem waits on its last one (previous iteration) when `wrap`.
// Within a stage slot the problems come in the order `rank` (grouped by
// filter length and blur radius, so that consecutive items run the same
// stage body and the instruction cache keeps it).
void order_stages(const std::vector<StageList>& per, const std::vector<int>& rank, bool wrap, int ctas,
                  std::vector<Stage>* out, std::vector<Item>* items) {
  size_t smax = 0;
  for (const auto& l : per) smax = std::max(smax, l.st.size());
  std::vector<int64_t> slot_tiles(smax, 0);
  for (const auto& l : per)
    for (size_t s = 0; s < l.st.size(); ++s) slot_tiles[s] += l.st[s].ntiles;
  std::vector<std::vector<int>> gidx(per.size());
  for (size_t p = 0; p < per.size(); ++p) gidx[p].assign(per[p].st.size(), -1);
  out->clear();
  for (size_t s = 0; s < smax; ++s)
    for (int p : rank)
      if (s < per[p].st.size()) {
        gidx[p][s] = static_cast<int>(out->size());
        Stage S = per[p].st[s];
        S.group = tiles_per_item(S, slot_tiles[s], ctas);
        out->push_back(S);
      }
  for (size_t p = 0; p < per.size(); ++p) {
    const size_t n = per[p].st.size();
    for (size_t s = 0; s < n; ++s) {
      Stage& S = (*out)[gidx[p][s]];
      if (s > 0) {
        S.prev = gidx[p][s - 1];
        S.prev_lag = 0;
      } else if (wrap) {
        S.prev = gidx[p][n - 1];
        S.prev_lag = 1;
      } else {
        S.prev = -1;
        S.prev_lag = 0;
      }
      S.prev_items = S.prev >= 0 ? stage_items((*out)[S.prev]) : 0;
    }
  }
  items->clear();
  for (size_t i = 0; i < out->size(); ++i) {
    const Stage& S = (*out)[i];
    const int g = S.group;
    for (int t = 0; t < S.ntiles; t += g) {
      Item it{};
      it.kind = S.kind;
      it.param = S.param;
      it.problem = S.problem;
      it.args = S.args;
      it.tiles_c = S.tiles_c;
      it.part = S.part;
      it.st = static_cast<int>(i);
      it.tile = t;
      it.prev = S.prev;
      it.pt2 = S.prev_items * 2 + S.prev_lag;
      it.ntl = std::min(g, S.ntiles - t);
      items->push_back(it);
    }
  }
}

Stage make_stage(int kind, int param, int problem, int args, int ntiles, int tiles_c, int part) {
  Stage s{};
  s.kind = kind;
  s.param = param;
  s.problem = problem;
  s.args = args;
  s.ntiles = ntiles;
  s.tiles_c = tiles_c;
  s.part = part;
  s.prev = -1;
  return s;
}

// a reconstruction level: 32 x 32 tiles, or 256-pixel items of the per-pixel
// gather for levels the tiles cannot fold (see the plan's generic_synth)
Stage syn_stage(const adjwt_wt_plan* w, int j, const SynArgs& a, int Lf, int p, int args) {
  if (w->lv[j - 1].generic_synth) {
    const int n = static_cast<int>(((int64_t)a.Nr * a.Nc + kGatherPixels - 1) / kGatherPixels);
    return make_stage(kGat, Lf, p, args, n, n, -1);
  }
  return make_stage(kSyn, Lf, p, args, a.tiles_c * a.tiles_r, a.tiles_c, -1);
}

template <typename T>
size_t put(std::vector<unsigned char>& blob, const std::vector<T>& v) {
  const size_t off = static_cast<size_t>(round_up(static_cast<int64_t>(blob.size()), 256));
  blob.resize(off + v.size() * sizeof(T) + 1);
  if (!v.empty()) std::memcpy(blob.data() + off, v.data(), v.size() * sizeof(T));
  return off;
}

int window_args(const adjwt_fista_problem& pr, const float* u, float* g, double* partials, BlurWinArgs* out) {
  std::memset(out, 0, sizeof(*out));
  out->a = blur_args(pr, u, g, partials);
  const adjwt_blur_plan* b = pr.blur;
  int uh, uw, vh, vw;
  window_boxes(blur_radius(b), &uh, &uw, &vh, &vw);
  int rc = make_tmap_2d_f32(&out->umap, u, b->rows, b->cols, b->image_pitch, uh, uw);
  if (!rc) rc = make_tmap_2d_f32(&out->bmap, pr.b, b->rows, b->cols, b->image_pitch, vh, vw);
  return rc;
}

size_t window_smem(int rmax) {
  switch (rmax) {
    case 2: return WG<2>::smem_bytes();
    case 3: return WG<3>::smem_bytes();
    case 4: return WG<4>::smem_bytes();
    case 5: return WG<5>::smem_bytes();
    case 6: return WG<6>::smem_bytes();
    case 7: return WG<7>::smem_bytes();
    case 8: return WG<8>::smem_bytes();
    case 9: return WG<9>::smem_bytes();
    default: return WG<12>::smem_bytes();
  }
}

// rmax_w / rmax_t: the largest padded radius of the problems whose blur stage
// takes the window tile / the gathered tile (0: none)
size_t engine_smem(int rmax_w, int rmax_t) {
  const int rmax = rmax_t;
  size_t blur = 0;
  if (rmax) switch (rmax) {
    case 2: blur = blur_tile_smem<2>(); break;
    case 3: blur = blur_tile_smem<3>(); break;
    case 4: blur = blur_tile_smem<4>(); break;
    case 5: blur = blur_tile_smem<5>(); break;
    case 6: blur = blur_tile_smem<6>(); break;
    case 7: blur = blur_tile_smem<7>(); break;
    case 8: blur = blur_tile_smem<8>(); break;
    case 9: blur = blur_tile_smem<9>(); break;
    default: blur = blur_tile_smem<12>(); break;
  }
  return std::max({kProxOffset + kProxSlotBytes, sizeof(SynSmem<10>), blur, rmax_w ? window_smem(rmax_w) : size_t{0}});
}

}  // namespace
}  // namespace adjwt

using namespace adjwt;

extern "C" size_t adjwt_fista_batch_workspace_size(int count, const adjwt_fista_problem* probs) {
  if (count <= 0 || !probs) return 0;
  size_t total = 0;
  for (int i = 0; i < count; ++i) {
    if (!probs[i].wt || !probs[i].blur) return 0;
    total += prob_ws(probs[i]).bytes;
  }
  return total;
}

extern "C" int adjwt_fista_batch_create(adjwt_fista_batch** out, int count, const adjwt_fista_problem* probs,
                                        float* const* x, float* const* y, void* ws, size_t ws_bytes) {
  if (!out) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_fista_batch_create: out is NULL");
  *out = nullptr;
  if (count < 1 || count > 65535 || !probs || !x || !y)
    return fail(ADJWT_ERR_INVALID_ARG, "adjwt_fista_batch_create: need 1 <= count <= 65535 and non-NULL arrays");
  for (int i = 0; i < count; ++i) {
    int rc = check_batch_problem(probs[i], i);
    if (rc) return rc;
    if (!x[i] || !y[i] || ((reinterpret_cast<uintptr_t>(x[i]) | reinterpret_cast<uintptr_t>(y[i])) & 15u))
      return fail(ADJWT_ERR_ALIGN, "adjwt_fista_batch_create: x and y must be non-NULL and 16-byte aligned");
  }
  const size_t need = adjwt_fista_batch_workspace_size(count, probs);
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < need)
    return fail(ADJWT_ERR_WORKSPACE, "adjwt_fista_batch_create: workspace of adjwt_fista_batch_workspace_size() "
                                     "bytes, 256-byte aligned, needed (" + std::to_string(need) + ")");
  auto* B = new adjwt_fista_batch();
  B->count = count;
  B->probs.assign(probs, probs + count);

  std::vector<SynArgs> syn;
  std::vector<AnaArgs> ana;
  std::vector<TiledArgs> blr;
  std::vector<BlurWinArgs> blw;
  std::vector<L1Args> l1;
  std::vector<ProbDev> pdev;
  std::vector<double*> moms;
  std::vector<StageList> run_lists(count), obj_lists(count);
  char* base = static_cast<char*>(ws);
  int rmax_w = 0, rmax_t = 0;
  for (int p = 0; p < count; ++p) {
    const adjwt_fista_problem& pr = probs[p];
    const adjwt_wt_plan* w = pr.wt;
    const ProbWs pw = prob_ws(pr);
    char* pb = base;
    base += pw.bytes;
    float* u = reinterpret_cast<float*>(pb + pw.u);
    float* g = reinterpret_cast<float*>(pb + pw.g);
    float* ll[2] = {reinterpret_cast<float*>(pb + pw.ll0), reinterpret_cast<float*>(pb + pw.ll1)};
    double* mom = reinterpret_cast<double*>(pb + pw.mom);
    double* parts = reinterpret_cast<double*>(pb + pw.parts);
    pdev.push_back(ProbDev{mom, parts, pw.nblur, pw.nl1, pr.lambda});
    moms.push_back(mom);
    const int J = w->levels, Lf = w->fb.L, R = blur_radius(pr.blur);
    const bool win = blur_window_ok(pr.blur);
    (win ? rmax_w : rmax_t) = std::max(win ? rmax_w : rmax_t, R);
    const int btc = blur_tiles_c(pr.blur);
    // the blur stage: kBlurW (TMA windows) or kBlur (gathered windows)
    auto blur_stage = [&](float* gout, double* parts_out, int part) -> Stage {
      if (win) {
        BlurWinArgs wa;
        if (window_args(pr, u, gout, parts_out, &wa)) return Stage{-1};
        blw.push_back(wa);
        return make_stage(kBlurW, R, p, static_cast<int>(blw.size()) - 1, pw.nblur, btc, part);
      }
      blr.push_back(blur_args(pr, u, gout, parts_out));
      return make_stage(kBlur, R, p, static_cast<int>(blr.size()) - 1, pw.nblur, btc, part);
    };
    // iteration: MOM, W levels J..1 on y, R^*(R u - b), W^* + prox levels 1..J
    auto& rl = run_lists[p].st;
    rl.push_back(make_stage(kMom, 0, p, 0, 1, 1, -1));
    for (int j = J; j >= 1; --j) {
      const SynArgs a = syn_level(w, j, y[p], u, ll);
      rl.push_back(syn_stage(w, j, a, Lf, p, static_cast<int>(syn.size())));
      syn.push_back(a);
    }
    rl.push_back(blur_stage(g, nullptr, -1));
    if (rl.back().kind < 0) {
      delete B;
      return fail(ADJWT_ERR_CUDA, "adjwt_fista_batch_create: tensor map encoding failed");
    }
    for (int j = 1; j <= J; ++j) {
      const AnaArgs a = ana_level(pr, j, g, x[p], y[p], ll, mom + 1);
      rl.push_back(make_stage(kAna, Lf, p, static_cast<int>(ana.size()), a.tiles_c * a.tiles_r, a.tiles_c, -1));
      ana.push_back(a);
    }
    // objective: W levels J..1 on x, 1/2 ||R u - b||^2 partials, |x| partials, the sum
    auto& ol = obj_lists[p].st;
    for (int j = J; j >= 1; --j) {
      const SynArgs a = syn_level(w, j, x[p], u, ll);
      ol.push_back(syn_stage(w, j, a, Lf, p, static_cast<int>(syn.size())));
      syn.push_back(a);
    }
    ol.push_back(blur_stage(nullptr, parts, 0));
    if (ol.back().kind < 0) {
      delete B;
      return fail(ADJWT_ERR_CUDA, "adjwt_fista_batch_create: tensor map encoding failed");
    }
    ol.push_back(make_stage(kL1, 0, p, static_cast<int>(l1.size()), pw.nl1, pw.nl1, pw.nblur));
    l1.push_back(L1Args{x[p], w->num_coeffs});
    ol.push_back(make_stage(kSum, 0, p, 0, 1, 1, -1));
  }
  std::vector<Stage> rst, ost;
  std::vector<Item> ritem, oitem;
  std::vector<int> rank(count);
  for (int p = 0; p < count; ++p) rank[p] = p;
  std::stable_sort(rank.begin(), rank.end(), [&](int a, int b) {
    const int ka = probs[a].wt->fb.L * 128 + blur_window_ok(probs[a].blur) * 64 + blur_radius(probs[a].blur);
    const int kb = probs[b].wt->fb.L * 128 + blur_window_ok(probs[b].blur) * 64 + blur_radius(probs[b].blur);
    return ka < kb;
  });
  // the launch's CTAs (resident ones: the grid never exceeds them)
  B->dyn = engine_smem(rmax_w, rmax_t);
  cudaError_t e = set_smem(k_fista_engine, B->dyn);
  int per_sm = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fista_engine, kEngineThreads, B->dyn);
  if (e != cudaSuccess) {
    delete B;
    return cuda_fail(e, "adjwt_fista_batch_create");
  }
  B->per_sm = std::max(per_sm, 1);
  const int ctas = B->per_sm * sm_count();
  order_stages(run_lists, rank, true, ctas, &rst, &ritem);
  order_stages(obj_lists, rank, false, ctas, &ost, &oitem);

  std::vector<unsigned char> blob;
  const size_t o_ritem = put(blob, ritem), o_oitem = put(blob, oitem);
  const size_t o_syn = put(blob, syn), o_ana = put(blob, ana), o_blr = put(blob, blr), o_l1 = put(blob, l1);
  const size_t o_blw = put(blob, blw);
  const size_t o_prob = put(blob, pdev), o_mom = put(blob, moms);
  const size_t nctr = kCtrDone + std::max(rst.size(), ost.size());
  const size_t o_ctr = static_cast<size_t>(round_up(static_cast<int64_t>(blob.size()), 256));
  B->counter_bytes = nctr * sizeof(int);
  const size_t total = o_ctr + B->counter_bytes;
  e = cudaMalloc(&B->dev, total);
  if (e == cudaSuccess) e = cudaMemcpy(B->dev, blob.data(), blob.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    delete B;
    return cuda_fail(e, "adjwt_fista_batch_create");
  }
  char* d = static_cast<char*>(B->dev);
  auto fill = [&](BatchLaunch& L, size_t oitem_, int nst, int items) {
    L.nstages = nst;
    L.items = items;
    L.args.items = reinterpret_cast<const Item*>(d + oitem_);
    L.args.items_per_iter = items;
    L.args.syn = reinterpret_cast<const SynArgs*>(d + o_syn);
    L.args.ana = reinterpret_cast<const AnaArgs*>(d + o_ana);
    L.args.blur = reinterpret_cast<const TiledArgs*>(d + o_blr);
    L.args.blurw = reinterpret_cast<const BlurWinArgs*>(d + o_blw);
    L.args.prob = reinterpret_cast<const ProbDev*>(d + o_prob);
    L.args.counters = reinterpret_cast<int*>(d + o_ctr);
    L.args.status = device_status_ptr();
  };
  fill(B->run, o_ritem, static_cast<int>(rst.size()), static_cast<int>(ritem.size()));
  fill(B->obj, o_oitem, static_cast<int>(ost.size()), static_cast<int>(oitem.size()));
  B->l1args = reinterpret_cast<const L1Args*>(d + o_l1);
  B->mom_ptrs = reinterpret_cast<double* const*>(d + o_mom);
  B->counters = reinterpret_cast<int*>(d + o_ctr);
  *out = B;
  return ADJWT_OK;
}

extern "C" void adjwt_fista_batch_destroy(adjwt_fista_batch* b) { delete b; }

namespace {
int set_momentum(const adjwt_fista_batch* b, double t, cudaStream_t s) {
  const unsigned nb = static_cast<unsigned>((b->count + 127) / 128);
  ADJWT_TRACED("fista_batch_reset", 0, s, pdl_launch(k_batch_reset, nb, 128, 0, s, b->mom_ptrs, b->count, t));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  return ADJWT_OK;
}
}  // namespace

extern "C" int adjwt_fista_batch_reset(const adjwt_fista_batch* b, adjwt_stream_t stream) {
  if (!b) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_fista_batch_reset: batch is NULL");
  return set_momentum(b, 1.0, static_cast<cudaStream_t>(stream));
}

extern "C" int adjwt_fista_batch_set_iteration(const adjwt_fista_batch* b, int64_t k, adjwt_stream_t stream) {
  if (!b) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_fista_batch_set_iteration: batch is NULL");
  if (k < 0 || k > 100000000) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_fista_batch_set_iteration: k outside 0..1e8");
  // t_{k+1} after k iterations from t_1 = 1, rounded as the device momentum stage does
  double t = 1.0, t1 = 0.0;
  float beta = 0.0f;
  for (int64_t i = 0; i < k; ++i) {
    fista_momentum(t, &t1, &beta);
    t = t1;
  }
  return set_momentum(b, t, static_cast<cudaStream_t>(stream));
}

namespace {
int engine_launch(const adjwt_fista_batch* b, const BatchLaunch& L, int iters, double* objectives, int stall,
                  cudaStream_t s, const char* name) {
  // tickets run up to two per CTA past the last item: keep them in int range
  if ((int64_t)L.items * iters > 0x7fffffff - (1 << 20))
    return fail(ADJWT_ERR_SHAPE, std::string(name) + ": iterations x items above 2^31 - 2^20");
  EngineArgs a = L.args;
  a.iters = iters;
  a.objectives = objectives;
  a.stall = stall;
  const int64_t total = (int64_t)L.items * iters;
  const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(total, (int64_t)b->per_sm * sm_count())));
  cudaError_t me = cudaSuccess;
  ADJWT_TRACED("fista_batch_reset_counters", 0, s, me = cudaMemsetAsync(b->counters, 0, b->counter_bytes, s));
  ADJWT_CUDA_CHECK(me);
  ADJWT_TRACED(name, 0, s, pdl_launch(k_fista_engine, dim3(grid), kEngineThreads, b->dyn, s, a, b->l1args));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  return ADJWT_OK;
}
}  // namespace

extern "C" int adjwt_fista_batch_run(const adjwt_fista_batch* b, int iters, adjwt_stream_t stream) {
  if (!b) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_fista_batch_run: batch is NULL");
  if (iters < 0) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_fista_batch_run: iters < 0");
  if (iters == 0) return ADJWT_OK;
  return engine_launch(b, b->run, iters, nullptr, 0, static_cast<cudaStream_t>(stream), "fista_batch");
}

extern "C" int adjwt_fista_batch_objective(const adjwt_fista_batch* b, double* objectives_dev, adjwt_stream_t stream) {
  if (!b || !objectives_dev) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_fista_batch_objective: NULL argument");
  return engine_launch(b, b->obj, 1, objectives_dev, 0, static_cast<cudaStream_t>(stream), "fista_batch_objective");
}

extern "C" int adjwt_fista_batch_wait_selftest(const adjwt_fista_batch* b, adjwt_stream_t stream) {
  if (!b) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_fista_batch_wait_selftest: batch is NULL");
  return engine_launch(b, b->run, 1, nullptr, 1, static_cast<cudaStream_t>(stream), "fista_batch_selftest");
}

extern "C" int adjwt_fista_batch_info(const adjwt_fista_batch* b, int* items_per_iteration, int* stages,
                                      int* ctas) {
  if (!b) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_fista_batch_info: batch is NULL");
  if (items_per_iteration) *items_per_iteration = b->run.items;
  if (stages) *stages = b->run.nstages;
  if (ctas) *ctas = b->per_sm * sm_count();
  return ADJWT_OK;
}
