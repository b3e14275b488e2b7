// Internal types shared by the host plan code and the CUDA kernels of libadjwt.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/adjwt.h"

namespace adjwt {

constexpr int kMaxLevels = 16;
constexpr int kMaxTaps = 10;     // longest filter array (CDF 9/7 in a length-10 array)
constexpr int kMaxBlurRadius = 32;
constexpr int kSynthTile = 32;   // output tile side of the tiled reconstruction kernel
constexpr int kChainCounterFloats = 64;  // level-chain counters at the tail of the second LL buffer

enum Mode : int { kZero = 0, kSym = 1, kPpd = 2, kPer = 3 };

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
#define ADJWT_CUDA_CHECK(call)                                  \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return ::adjwt::cuda_fail(e_, #call); \
  } while (0)

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// Programmatic dependent launch.  Every kernel of this library is launched
// with programmatic stream serialisation and starts with pdl_entry(): it lets
// the next kernel in the stream begin launching once all of its own CTAs are
// resident, then waits until the preceding kernel has completed and its
// writes are visible.  Chains of small dependent kernels (the deep wavelet
// levels) thereby hide their launch latency.  Nothing is read or written
// before the wait.
#if defined(__CUDACC__)
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
#endif

// Whether (kernel, current device) already has at least `bytes` of dynamic
// shared memory enabled; records it when `mark` is set.
bool smem_attr_known(const void* kernel, size_t bytes, bool mark);

// Opt a kernel into `bytes` of dynamic shared memory and the largest shared
// carveout, so that several such CTAs can be resident on one SM.  Done once
// per kernel and device, so that later launches (e.g. under stream capture)
// make no attribute calls.
template <typename Kernel>
inline cudaError_t set_smem(Kernel kernel, size_t bytes) {
  const void* key = reinterpret_cast<const void*>(kernel);
  if (smem_attr_known(key, bytes, false)) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e == cudaSuccess) smem_attr_known(key, bytes, true);
  return e;
}

// ---------------------------------------------------------------- device status, TMA descriptors
// Address of the device status word of the current device (null on failure).
int* device_status_ptr();
// 2D float32 tensor map over rows x cols (row pitch in floats) with a
// box_rows x box_cols box; out-of-range elements read as zero.
int make_tmap_2d_f32(CUtensorMap* map, const float* base, int rows, int cols, int pitch_floats, int box_rows,
                     int box_cols);
// The same with the 128-byte swizzle (box rows of 128 bytes; the shared-memory
// box must start 1024-byte aligned): 16-byte chunk c of box row r lies at
// chunk position c ^ (r mod 8).
int make_tmap_2d_f32_sw(CUtensorMap* map, const float* base, int rows, int cols, int pitch_floats, int box_rows,
                        int box_cols, bool swizzle128);
int sm_count();

// ---------------------------------------------------------------- tracing
int trace_begin(const char* name, int tag, cudaStream_t s);     // level 1: one kernel
int trace_op_begin(const char* name, int tag, cudaStream_t s);  // level 2: one operator call
void trace_end(int id, cudaStream_t s);
#define ADJWT_TRACED(name, tag, stream, ...)                      \
  do {                                                            \
    const int tr_id_ = ::adjwt::trace_begin(name, tag, stream);   \
    __VA_ARGS__;                                                  \
    ::adjwt::trace_end(tr_id_, stream);                           \
  } while (0)
#define ADJWT_TRACED_OP(name, tag, stream, ...)                     \
  do {                                                              \
    const int tr_op_ = ::adjwt::trace_op_begin(name, tag, stream);  \
    __VA_ARGS__;                                                    \
    ::adjwt::trace_end(tr_op_, stream);                             \
  } while (0)

// ---------------------------------------------------------------- filters
struct FilterBank {
  int L = 0;
  double dec_lo[kMaxTaps] = {}, dec_hi[kMaxTaps] = {}, rec_lo[kMaxTaps] = {}, rec_hi[kMaxTaps] = {};
};
bool make_filter_bank(int wavelet, FilterBank* fb);

// ---------------------------------------------------------------- wavelet plan
// One axis of one level.
struct LevelAxis {
  int N;          // length of LL_{j-1} along this axis (level input)
  int n;          // band length along this axis
  int pitch_in;   // unused for axis 1 / rows
  const float* winv;  // device table of 1/c[j], j < N (null for PER / ZERO)
};

struct Level {
  LevelAxis ax[2];  // 0 = rows (vertical), 1 = cols (horizontal)
  int in_pitch;     // row pitch of LL_{j-1} (image pitch for j = 1)
  int band_pitch;   // row pitch of the four bands of level j
  int64_t off_band[4];  // offsets of LL(level J only) / LH / HL / HH in the packed vector (-1 = none)
  bool generic_synth;   // synthesis of this level takes the per-pixel gather path
};

}  // namespace adjwt

struct adjwt_wt_plan {
  int rows, cols, levels, wavelet, bc;
  adjwt::FilterBank fb;
  int image_pitch;
  int64_t num_coeffs;
  std::vector<int64_t> band_offsets;  // 3J+1 packed order
  std::vector<int> band_rows, band_cols, band_pitch;
  std::vector<adjwt::Level> lv;       // lv[j-1] = level j
  int64_t ll_buf_floats[2];           // ping-pong LL buffer sizes (odd / even levels)
  float* d_tables = nullptr;          // device copy of all 1/c tables
  // per operator (0: W, 1: W^* and W^dagger, 2: W^* with the FISTA prox
  // epilogue) and level: 1 = the level runs on the tiled kernel alone, 0 = the
  // TMA kernel takes the tiles the size rule gives it (set by
  // adjwt_wt_plan_set_tma / adjwt_wt_plan_autotune)
  unsigned char tma_off[3][adjwt::kMaxLevels] = {};
  // resident CTAs per SM of the persistent TMA kernel per operator and level
  // (0: as many as fit); the autotuner's second axis
  unsigned char tma_ctas[3][adjwt::kMaxLevels] = {};
  // the deepest run of tiled-only levels runs as one level-chain launch only
  // when switched on (adjwt_wt_plan_set_level_chain); off by default
  bool chain_off = true;
};

struct adjwt_blur_plan {
  int rows, cols, bc, kr, kc, image_pitch;
  double taps_r[2 * adjwt::kMaxBlurRadius + 1], taps_c[2 * adjwt::kMaxBlurRadius + 1];
};

namespace adjwt {

// ---------------------------------------------------------------- launchers (stream-ordered)
struct ProxArgs {
  float* x;          // packed coefficient buffers (state), null = plain W^* output
  float* y;
  float step;        // 1/L_f
  float thresh;      // lambda/L_f
  float beta;        // (t_k - 1)/t_{k+1}
  double* l1_partials;  // per-CTA partial sums of |x_k| (null = skip)
  const double* beta_dev;  // non-null: momentum factor read from device memory instead of beta
};

// W (wt_synth): coeffs -> image.  ws holds the LL ping-pong buffers.
int launch_wt_synth(const adjwt_wt_plan* p, const float* coeffs, float* image, float* llbuf0, float* llbuf1,
                    cudaStream_t s);
// Analysis direction: W^* (adjoint = true) or W^dagger.  With prox.x != null
// the final bands are not written to `coeffs` but fed to the FISTA prox step.
int launch_wt_analysis(const adjwt_wt_plan* p, const float* image, float* coeffs, bool adjoint,
                       const ProxArgs& prox, float* llbuf0, float* llbuf1, cudaStream_t s, int* l1_slots_used);
int wt_l1_partial_slots(const adjwt_wt_plan* p);
// First level of the level chain (levels j0..J in one launch) of the
// analysis direction (W^*, W^dagger; prox: W^* with the FISTA prox) and of
// the reconstruction W; levels + 1 when the transform has none.
int ana_chain_start(const adjwt_wt_plan* p, bool adjoint, bool prox);
int syn_chain_start(const adjwt_wt_plan* p);
// Interior rectangle of level j's output reconstructed by the persistent TMA
// kernel (empty for small levels), and its launcher.
void synth_tma_rect(const adjwt_wt_plan* p, int j, int* r0, int* r1, int* c0, int* c1);
int launch_synth_tma(const adjwt_wt_plan* p, int j, const float* const band[4], float* out, int out_pitch,
                     cudaStream_t s);
// Whether level j of the analysis direction (W^*, optionally with the prox,
// or W^dagger) runs whole on the persistent TMA analysis kernel, and its
// launcher; *ncta receives the number of l1 partial slots it wrote.
bool ana_tma_level(const adjwt_wt_plan* p, int j, bool prox);
int launch_ana_tma(const adjwt_wt_plan* p, int j, bool adjoint, const float* in, int in_pitch, float* const dst[4],
                   float* const px[4], float* const py[4], int out_pitch, float step, float thresh, float beta,
                   const double* beta_dev, double* l1, const float* flo, const float* fhi, const char* name,
                   cudaStream_t s, int* ncta);

// Blur family.
int launch_blur(const adjwt_blur_plan* p, const float* in, float* out, bool adjoint, cudaStream_t s);
// Fused R^*(R u - b).  With an image-sized scratch buffer v and a radius
// <= 12 it runs as two persistent TMA-staged passes (v = R u - b, g = R^* v);
// otherwise as one tiled kernel.  *nparts receives the number of float64
// partials written.
int launch_blur_normal(const adjwt_blur_plan* p, const float* u, const float* b, float* g, double* partials,
                       float* scratch_v, cudaStream_t s, int* nparts);
size_t blur_partials_bytes(const adjwt_blur_plan* p);
// Persistent TMA-staged single pass (radius <= 12): R u (- b, partials) or R^* v.
bool tma_blur_supported(const adjwt_blur_plan* p);
int tma_blur_partial_slots(const adjwt_blur_plan* p);
int launch_tma_blur(const adjwt_blur_plan* p, bool adjoint, const float* in, const float* b, float* out,
                    double* partials, cudaStream_t s, int* nparts);
int launch_blur_residual_norm(const adjwt_blur_plan* p, const float* u, const float* b, double* partials,
                              cudaStream_t s, int* nparts);
int blur_partial_slots(const adjwt_blur_plan* p);
// Register-blocked fused R^*(R u - b) tiles for radii <= 12, no scratch.
bool tiled_blur_supported(const adjwt_blur_plan* p);
int tiled_blur_grid_slots(const adjwt_blur_plan* p);
int launch_tiled_blur(const adjwt_blur_plan* p, const float* in, const float* b, float* out, double* partials,
                      cudaStream_t s);

// FISTA momentum: t_{k+1} and the float32 extrapolation weight beta_k.
void fista_momentum(double t, double* t_next, float* beta);

// Deterministic sum of float64 partials: out[0] = scale0 * sum(a[0..na)) + scale1 * sum(b[0..nb)).
int launch_sum_partials(const double* a, int na, double scale_a, const double* b, int nb, double scale_b,
                        double* out, cudaStream_t s);

// Differentiation pieces (grad.cu): out = a x + b y on rows x cols of pitched
// arrays; float64 per-block partials of an inner product and of the soft
// threshold's sum sign(x_next) xbar (zbar = xbar where x_next != 0), with
// *nparts partials written (at most reduce_partials_bytes() / 8).
int launch_axpby(int rows, int64_t cols, int64_t pitch, float a, const float* x, float b, const float* y, float* out,
                 cudaStream_t st);
int launch_dot_partials(int rows, int64_t cols, int64_t pitch, const float* x, const float* y, double* partials,
                        cudaStream_t st, int* nparts);
int launch_prox_vjp_partials(int64_t n, const float* x_next, const float* xbar, float* zbar, double* partials,
                             cudaStream_t st, int* nparts);
size_t reduce_partials_bytes();

// Tuning cache: apply the stored per-level TMA choices of this plan's size
// class (rows, cols, levels, wavelet, boundary, device), if any.
void apply_tuning_cache(adjwt_wt_plan* p);

// Convolution family.
int launch_conv_adjoint(int batch, int64_t n, int k, const float* s, const float* h, const float* r,
                        float* grad_h, float* grad_s, float* partials, cudaStream_t st);
int64_t conv_partial_floats(int batch, int64_t n, int k);
int64_t conv_static_scratch_floats();
void conv_reduce(unsigned nblocks, int k, int nchunks, const float* partials, float* grad_h, int64_t total,
                 cudaStream_t st);
// Register-blocked channel-gradient kernel (k <= 1024): r given (r_in) or
// computed as h * s - x in the same pass.
bool conv_fused_supported(int k);
int64_t conv_fused_nchunks(int64_t n, int k);
int launch_conv_fused(int batch, int64_t n, int k, const float* s, const float* h, const float* x, const float* r_in,
                      float* r_out, float* grad_h, float* grad_s, float* partials, cudaStream_t st);
// Tensor-core channel-gradient kernel for 49 <= k <= 64 (tcgen05 TF32 with a
// float32-accurate three-product split); launch_conv_fused routes those k here
// unless ADJWT_CONV_FP32 is set to a non-zero value in the environment.  Its
// grad_h partials need at most as many slots as the register-blocked kernel's.
bool conv_tc_supported(int k);
int64_t conv_tc_nchunks(int64_t n);
int launch_conv_tc(int batch, int64_t n, int k, const float* s, const float* h, const float* x, const float* r_in,
                   float* r_out, float* grad_h, float* grad_s, float* partials, cudaStream_t st);
int launch_conv_adjoint_noalloc(int batch, int64_t n, int k, const float* s, const float* h, const float* r,
                                float* grad_h, float* grad_s, cudaStream_t st);
int launch_conv_residual(int batch, int64_t n, int k, const float* h, const float* s, const float* x, float* r,
                         cudaStream_t st);
// Eq. 6: grad_h <- 2 grad_h + (lambda_tv/delta) D^T clip(D h), grad_s = 2 sum_c gs_rows[c].
int launch_bce_finish(int C, int64_t n, int k, const float* h, float* grad_h, const float* gs_rows, float* grad_s,
                      double lambda_tv, double delta, cudaStream_t s);


}  // namespace adjwt
