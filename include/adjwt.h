/*
 * adjwt -- exact adjoints of multi-level 2D wavelet reconstruction and of
 * Gaussian blur, the FISTA gradient W^* R^* (R W x - b) built from them, and
 * the blind-channel convolution adjoint, on one GB300 (sm_103a).
 *
 * Paper: J. Folberth, S. Becker, "Efficient Adjoint Computation for Wavelet
 * and Convolution Operators", IEEE Signal Processing Magazine (Lecture
 * Notes), arXiv 1707.02018.
 *
 * Conventions for every entry point
 *  - Tensors are caller-owned DEVICE buffers of float32 unless stated.
 *    Pointers must be 16-byte aligned.  Calls are asynchronous on `stream`
 *    except where a host result is returned (stated per call).
 *  - Images are rows x cols, row-major, with a row pitch of image_pitch
 *    floats (cols rounded up to a multiple of 4).  Pitch padding of an image
 *    is ignored on input and left untouched on output.
 *  - Coefficient vectors use the packed band order
 *      [LL_J, LH_J, HL_J, HH_J, LH_{J-1}, ..., HH_1]
 *    (LH = vertical highpass / horizontal lowpass, HL = vertical lowpass /
 *    horizontal highpass).  Band b is band_rows[b] x band_cols[b] with row
 *    pitch band_pitch[b] (multiple of 4 floats) starting at band_offsets[b]
 *    floats; num_coeffs counts the padding.  Padding is ignored on input and
 *    written as 0 on output.
 *  - Plans are created once (they allocate a few KB of device tables), are
 *    immutable apart from the level-implementation switches of wavelet
 *    plans (set before use), and may be used concurrently from several
 *    streams.  Hot calls
 *    allocate nothing: scratch comes from a caller-provided workspace of at
 *    least *_workspace_size bytes (256-byte aligned).
 *  - Out-of-place only: an output that overlaps an input -> ADJWT_ERR_ALIAS.
 *  - Return 0 on success or a negative ADJWT_ERR_* code; adjwt_last_error()
 *    then holds a message for the calling thread.  Nothing throws or aborts
 *    across this boundary.
 */
#ifndef ADJWT_H
#define ADJWT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* adjwt_stream_t; /* same type as cudaStream_t */

enum {
  ADJWT_OK = 0,
  ADJWT_ERR_INVALID_ARG = -1, /* null pointer, unknown enum, bad scalar     */
  ADJWT_ERR_SHAPE = -2,       /* sizes unsupported for this mode            */
  ADJWT_ERR_ALIGN = -3,       /* pointer not 16-byte aligned                */
  ADJWT_ERR_ALIAS = -4,       /* output overlaps an input                   */
  ADJWT_ERR_CUDA = -5,        /* CUDA runtime error (text in last_error)    */
  ADJWT_ERR_NONFINITE = -6,   /* objective or step size not finite          */
  ADJWT_ERR_WORKSPACE = -7,   /* workspace missing, small or misaligned     */
  ADJWT_ERR_TIMEOUT = -8,     /* a bounded device wait gave up              */
  ADJWT_ERR_BOUNDS = -9       /* checked builds only (-DADJWT_BOUNDS_CHECK):
                                 a device access fell outside its buffer; it
                                 was skipped and recorded in the status word */
};

/* Boundary handling (Sec. I-A).  ZERO: zero-padded extension E_zpd.  SYM:
 * half-point symmetric E_sym.  PPD: the periodic extension E_per of Sec. I-A
 * (redundant).  PER: critically sampled circular transform (sizes divisible by
 * 2^levels; for orthogonal filters W^* = W^-1).  Blur plans take ZERO, SYM or
 * PER (PER = circular wrap). */
typedef enum { ADJWT_BC_ZERO = 0, ADJWT_BC_SYM = 1, ADJWT_BC_PPD = 2, ADJWT_BC_PER = 3 } adjwt_bc;

/* Filter banks (Sec. I-B orthogonal Haar / Daubechies, Sec. I-C CDF 9/7).
 * DB2 = 4-tap Daubechies, DB4 = 8-tap, CDF97 = 9/7 biorthogonal in a length-10
 * array.  L = 2, 4, 8, 10; extension length per side L' = L - 1. */
typedef enum { ADJWT_HAAR = 0, ADJWT_DB2 = 1, ADJWT_DB4 = 2, ADJWT_CDF97 = 3 } adjwt_wavelet;

typedef struct adjwt_wt_plan adjwt_wt_plan;
typedef struct adjwt_blur_plan adjwt_blur_plan;

/* Message of the last failed call on this thread ("" if none). */
const char* adjwt_last_error(void);
int adjwt_version(void);

/* Device status word of the current device.  Kernels that stage tiles with
 * the TMA unit bound every wait on an asynchronous copy (about one second);
 * one that gives up records ADJWT_ERR_TIMEOUT here and returns without
 * writing its outputs.  Reads the word into *status_out (0 = no failure)
 * after synchronising the device, and resets it to 0 when clear != 0. */
int adjwt_device_status(int* status_out, int clear);

/* Exercises that bounded wait without any fault: one thread arms a barrier
 * that expects one arrival and waits on it exactly as the staging kernels
 * do.  arrive != 0: it arrives itself and the wait ends at once.  arrive == 0:
 * nothing completes the barrier, the wait gives up after its limit (about one
 * second) and the kernel records ADJWT_ERR_TIMEOUT in the device status word
 * and returns; the context stays usable.  Asynchronous on `stream`; read the
 * result with adjwt_device_status.  No counterpart in the paper. */
int adjwt_wait_selftest(int arrive, adjwt_stream_t stream);

/* ------------------------------------------------------------------ wavelets
 * Plan of a J-level 2D transform of a rows x cols image.  Band lengths per
 * level and axis: n = floor((N + 3L')/2) for ZERO/SYM/PPD (the full
 * zero-padded analysis of the length N + 2L' extended signal, odd samples),
 * n = N/2 for PER.  rows, cols >= 1; 1 <= levels <= 16.
 * Errors: INVALID_ARG (enum), SHAPE (PER sizes not divisible by 2^levels),
 * CUDA (table allocation). */
int adjwt_wt_plan_create(adjwt_wt_plan** out, int rows, int cols, int levels, int wavelet, int bc);
void adjwt_wt_plan_destroy(adjwt_wt_plan* plan);

/* Layout of the packed coefficient vector.  Arrays hold 3*levels+1 entries in
 * packed band order; any output pointer may be NULL. */
int adjwt_wt_layout(const adjwt_wt_plan* plan, int64_t* num_coeffs, int64_t* band_offsets,
                    int* band_rows, int* band_cols, int* band_pitch, int* image_pitch);

/* Workspace bytes needed by wt_synth / wt_synth_adjoint / wt_analysis. */
size_t adjwt_wt_workspace_size(const adjwt_wt_plan* plan);

/* The filter taps the plan derived (float64, length L each; NULL skips). */
int adjwt_wt_filters(const adjwt_wt_plan* plan, double* dec_lo, double* dec_hi, double* rec_lo,
                     double* rec_hi, int* L);

/* W: multi-level reconstruction, W = E^dagger W_zpd per level (Sec. I-A,
 * Eq. 2 with W^dagger = W^dagger_zpd E): coeffs (num_coeffs) -> image. */
int wt_synth(const adjwt_wt_plan* plan, const float* coeffs, float* image, void* ws, size_t ws_bytes,
             adjwt_stream_t stream);

/* W^*: the exact adjoint of wt_synth, Eq. 4: dual-filter zero-padded analysis
 * after the weighted extension (E^dagger)^*: image -> coeffs. */
int wt_synth_adjoint(const adjwt_wt_plan* plan, const float* image, float* coeffs, void* ws,
                     size_t ws_bytes, adjwt_stream_t stream);

/* W^dagger: analysis W^dagger_zpd E (Sec. I-A); wt_synth(wt_analysis(u)) = u.
 * The "pseudoinverse approximation" of W^* discussed in Sec. I-B. */
int wt_analysis(const adjwt_wt_plan* plan, const float* image, float* coeffs, void* ws, size_t ws_bytes,
                adjwt_stream_t stream);

/* Level implementations.  A level of W (op 0), of W^* / W^dagger (op 1) or
 * of W^* with the FISTA prox epilogue (op 2, a kernel of its own: it also
 * reads and writes the iterate) runs either on a persistent TMA-staged
 * kernel or on the tiled kernel alone.  Size rule: for W the TMA kernel
 * takes whole levels of at least 256 x 512 whose tiles need no fold (ZERO,
 * PER) and, from 1536 x 1536, the interior tiles of any level, the tiled
 * kernel doing the border; for W^* it takes every tile of levels of at least
 * 1536 x 1536 (border windows completed in shared memory).  Results agree
 * within float32 rounding either way.  adjwt_wt_plan_set_tma(plan, op,
 * level, 0) forces the tiled kernel for that level, 1 restores the rule;
 * adjwt_wt_plan_uses_tma reports whether the TMA kernel runs there.
 * adjwt_wt_plan_set_tma_ctas(plan, op, level, c) caps the persistent TMA
 * kernel of that level at c resident CTAs per SM (c = 1..3; 0, the default:
 * as many as fit), which trades latency hiding for longer per-CTA copy
 * pipelines; adjwt_wt_plan_tma_ctas reads the setting.
 * adjwt_wt_plan_autotune measures: for every level the rule makes eligible
 * it times `reps` whole transforms (W, W^*, then W^* with the prox on
 * scratch iterates) with the level on each of four candidates (the tiled
 * kernel alone; the TMA kernel with as many CTAs per SM as fit, with one,
 * with two), keeps another candidate than the default (the TMA kernel, as
 * many CTAs as fit) only if it is at least 3 % faster, and stores the
 * choices for the plan's size class (rows, cols, levels, wavelet, boundary,
 * current device);
 * plans created later for that class start from them, and autotuning such a
 * class again only applies them (*from_cache = 1; from_cache may be NULL).
 * It allocates and frees its own device buffers and synchronises the
 * stream.  These calls change the plan: make them before the plan is used
 * on other streams.  Errors: INVALID_ARG (op outside 0..2, reps outside
 * 1..1000, ctas outside 0..3, NULL), SHAPE (level outside 1..levels), CUDA. */
int adjwt_wt_plan_set_tma(adjwt_wt_plan* plan, int op, int level, int enabled);
int adjwt_wt_plan_uses_tma(const adjwt_wt_plan* plan, int op, int level, int* uses);
int adjwt_wt_plan_set_tma_ctas(adjwt_wt_plan* plan, int op, int level, int ctas);
int adjwt_wt_plan_tma_ctas(const adjwt_wt_plan* plan, int op, int level, int* ctas);
int adjwt_wt_plan_autotune(adjwt_wt_plan* plan, int reps, int* from_cache, adjwt_stream_t stream);

/* Level chain (no counterpart in the paper: a launch schedule).  The deepest
 * run of at least two levels that the TMA kernel does not share (for W also
 * none on the per-pixel gather path, and never under PPD) runs as ONE launch
 * instead of one launch per level: its tiles are items handed out level by
 * level in the order of the recursion (Eq. 2 / Eq. 4: W^* from level 1 down,
 * W from level J up), and a tile starts once every tile of the level it reads
 * is done.  Its counters live in the workspace and are zeroed on the stream
 * before each launch; waits are bounded (ADJWT_ERR_TIMEOUT in the device
 * status word).  Results are identical to the per-level launches.  It is
 * OFF by default: on GB300 it measured slower than the per-level launches
 * (whose launch latency programmatic dependent launch already hides), e.g.
 * 2048^2 5-level CDF 9/7 W 89 vs 64 us, 256^2 3-level db2 W 31 vs 25 us.
 * adjwt_wt_plan_set_level_chain(plan, 1) switches it on (0: off);
 * adjwt_wt_plan_chain_start gives the chain's first level for op 0 (W), 1
 * (W^*) or 2 (W^* with the prox), 0 when that transform has none (or the
 * chain is off).
 * Errors: INVALID_ARG (NULL, op outside 0..2). */
int adjwt_wt_plan_set_level_chain(adjwt_wt_plan* plan, int enabled);
int adjwt_wt_plan_chain_start(const adjwt_wt_plan* plan, int op, int* first_level);

/* ---------------------------------------------------------------------- blur
 * Separable PSF p = outer(taps_r, taps_c) (float64 taps, odd lengths
 * kr, kc <= 65) applied as R u = C_valid(E_r u) under bc in {ZERO, SYM, PER}
 * (Sec. I: Gaussian PSF under symmetric boundary conditions).  Images use
 * image_pitch = cols rounded up to 4. */
int adjwt_blur_plan_create(adjwt_blur_plan** out, int rows, int cols, const double* taps_r, int kr,
                           const double* taps_c, int kc, int bc);
void adjwt_blur_plan_destroy(adjwt_blur_plan* plan);
int adjwt_blur_image_pitch(const adjwt_blur_plan* plan);
/* Workspace of blur_normal: float64 partial sums followed by one image-sized
 * scratch buffer holding R u - b between the two passes. */
size_t adjwt_blur_workspace_size(const adjwt_blur_plan* plan);

/* out = R in. */
int blur(const adjwt_blur_plan* plan, const float* in, float* out, adjwt_stream_t stream);
/* out = R^* in = E_r^T C_valid^T in (correlation, then fold the extension). */
int blur_adjoint(const adjwt_blur_plan* plan, const float* in, float* out, adjwt_stream_t stream);
/* Image-space data gradient g = R^*(R u - b) (the residual step of Sec. I);
 * if half_sq_out (DEVICE double) is non-NULL it receives 1/2 ||R u - b||^2
 * (float32 per thread, float64 across threads).  b may be NULL (taken as 0).
 * With a workspace of adjwt_blur_workspace_size bytes (required when
 * half_sq_out is set) and PSF radii <= 12, it runs as two TMA-staged passes
 * through the scratch image; with ws == NULL, as one fused tiled kernel. */
int blur_normal(const adjwt_blur_plan* plan, const float* u, const float* b, float* g, double* half_sq_out,
                void* ws, size_t ws_bytes, adjwt_stream_t stream);

/* ------------------------------------------------------- blind channel (Sec. II)
 * Batched real signals, row-major with unit stride: s (batch x n),
 * h (batch x k), r and x (batch x (n+k-1)).  Eq. 5 gradients:
 *   grad_h[b][j] = sum_{i<n} s[b][i] r[b][i+j]   (j < k)   = S^T r
 *   grad_s[b][m] = sum_{i<k} h[b][i] r[b][i+m]   (m < n)   = H^T r
 * either output may be NULL.  batch >= 0, n >= 1, k >= 1.  Channels of
 * 49..64 taps run on the tensor cores (TF32 operands split into high and low
 * parts, float32-accurate); other lengths on the CUDA cores.  Setting the
 * environment variable ADJWT_CONV_FP32 to a non-zero value before the first
 * call sends every k <= 1024 to the CUDA-core kernel. */
size_t adjwt_conv_adjoint_workspace_size(int batch, int64_t n, int k);
int conv_adjoint(int batch, int64_t n, int k, const float* s, const float* h, const float* r, float* grad_h,
                 float* grad_s, void* ws, size_t ws_bytes, adjwt_stream_t stream);
/* Both gradients of Eq. 5 at (h, s) in one pass: r = h * s - x (full
 * convolution, x of length n+k-1, NULL = 0) is formed on chip and fed to
 * grad_h = S^T r and grad_s = H^T r; r is also written out when r != NULL.
 * Any of r, grad_h, grad_s may be NULL.  Workspace:
 * adjwt_conv_gradient_workspace_size (it holds r too when k > 1024). */
size_t adjwt_conv_gradient_workspace_size(int batch, int64_t n, int k);
int conv_gradient(int batch, int64_t n, int k, const float* s, const float* h, const float* x, float* r,
                  float* grad_h, float* grad_s, void* ws, size_t ws_bytes, adjwt_stream_t stream);

/* conv_adjoint without a workspace argument (the paper has no counterpart;
 * this is a deployment variant).  It is for callers that must not allocate
 * device memory on their call path: processes whose device memory is owned by
 * another allocator (a framework's pool, a fixed budget), loops in which the
 * device-wide synchronisation of cudaMalloc/cudaFree is not acceptable, and
 * deployments that forbid allocation after start-up.  The grad_h partial sums
 * go to a fixed 4 MiB array (2^20 floats) in the library's device memory,
 * which every GPU that loads the library holds until the process exits; the
 * call itself allocates nothing.  Limit: when grad_h is requested,
 * batch * ceil(n / c) * k <= 2^20 with the chunk
 * c = 16 * floor((4097 - 16 * ceil(k / 16)) / 16) for k <= 1024 (c = 4032 at
 * k = 64, 3072 at k = 1024) and c = 1024 above, else
 * ADJWT_ERR_WORKSPACE and nothing runs.  (For 49 <= k <= 64 the tensor-core
 * kernel runs with 4096-sample chunks and so uses no more than this bound.)
 * The first call in a context looks up the array's device address (with the
 * device current) and caches it under the context's process-unique id: the
 * address is tied to the context, and a new context (after cudaDeviceReset,
 * or a non-primary context made current) gets its own lookup.  Make the first
 * call in each context before any stream capture.  All calls share the array: calls that overlap on the GPU (other
 * streams, other threads) race and must be serialised by the caller.
 * Results equal conv_adjoint's; arguments, layouts and errors as there. */
int conv_adjoint_noalloc(int batch, int64_t n, int k, const float* s, const float* h, const float* r,
                         float* grad_h, float* grad_s, adjwt_stream_t stream);

/* Residual of the full convolution, r = h * s - x (x may be NULL: r = h * s). */
int conv_residual(int batch, int64_t n, int k, const float* h, const float* s, const float* x, float* r,
                  adjwt_stream_t stream);

/* Gradient of the smooth part of the augmented multichannel problem of
 * Sec. II, Eq. 6: `channels` responses h_c (channels x k) share the source s
 * (length n); observations x (channels x (n+k-1)); r_c = h_c * s - x_c;
 *   f = sum_c ||r_c||^2 + (lambda_tv/delta) L_delta(D h_c),  (D h)[j] = h[j+1]-h[j],
 *   grad_h[c] = 2 S^T r_c + (lambda_tv/delta) D^T clip(D h_c, -delta, delta),
 *   grad_s    = sum_c 2 H_c^T r_c   (L_delta = Huber, clip = its derivative).
 * Either output may be NULL.  delta > 0, lambda_tv >= 0 (INVALID_ARG);
 * channels, n, k >= 1 and k <= 4096 (SHAPE).  Workspace:
 * adjwt_bce_gradient_workspace_size bytes, 256-byte aligned. */
size_t adjwt_bce_gradient_workspace_size(int channels, int64_t n, int k);
int bce_gradient(int channels, int64_t n, int k, const float* s, const float* h, const float* x, double lambda_tv,
                 double delta, float* grad_h, float* grad_s, void* ws, size_t ws_bytes, adjwt_stream_t stream);

/* --------------------------------------------------------------------- FISTA
 * min_x 1/2 ||R W x - b||^2 + lambda ||x||_1 (Eq. 1) with constant step
 * 1/lipschitz.  The wavelet and blur plans must describe the same image. */
typedef struct {
  const adjwt_wt_plan* wt;
  const adjwt_blur_plan* blur;
  const float* b;   /* device image (observed, blurred) */
  double lambda;    /* > 0 */
  double lipschitz; /* L_f > 0, e.g. from adjwt_fista_lipschitz */
  int gradient;     /* ADJWT_GRAD_ADJOINT (0): grad f = W^* R^*(R W y - b);
                       ADJWT_GRAD_PINV (1): W^dagger in place of W^*, the
                       substitute the paper compares against (Sec. I-B, I-C) */
} adjwt_fista_problem;

enum { ADJWT_GRAD_ADJOINT = 0, ADJWT_GRAD_PINV = 1 };

typedef struct {
  float* x;  /* device coeffs: x_{k-1} on entry, x_k on return       */
  float* y;  /* device coeffs: y_k on entry, y_{k+1} on return       */
  double t;  /* t_k on entry (1 before the first step), t_{k+1} on return */
  int64_t k; /* number of steps taken                                 */
} adjwt_fista_state;

size_t adjwt_fista_workspace_size(const adjwt_fista_problem* prob);

/* One FISTA iteration (the method cited in Sec. I-B):
 *   x_k = soft(y_k - grad f(y_k)/L_f, lambda/L_f),  grad f = W^* R^*(R W y_k - b)
 *   t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2,  y_{k+1} = x_k + ((t_k-1)/t_{k+1})(x_k - x_{k-1}).
 * If objective_out (HOST) is non-NULL the call also evaluates F(x_k) and
 * synchronises the stream; a non-finite value returns ADJWT_ERR_NONFINITE. */
int fista_step(const adjwt_fista_problem* prob, adjwt_fista_state* state, void* ws, size_t ws_bytes,
               double* objective_out, adjwt_stream_t stream);

/* Batched FISTA engine (the batching extension; the paper solves one
 * problem at a time).  Many independent problems (Eq. 1, each with its own
 * plans, observation, lambda, L_f and gradient mode) advance `iters` FISTA
 * iterations in ONE persistent kernel launch: the work is cut into items of
 * one stage of one problem (stages: the momentum update, W level J..1, the
 * fused R^*(R u - b), W^* + prox level 1..J; tiles of 32 x 32 wavelet
 * outputs and 32 x 64 blur outputs, 64 x 64 under SYM with non-palindromic
 * taps; an item is one tile, or two to four consecutive tiles when the
 * batch holds far more tiles than the launch has CTAs), numbered
 * stage-major across problems and taken by
 * the CTAs in order; a stage starts once the previous stage of its problem
 * is done.  Waits are bounded (ADJWT_ERR_TIMEOUT in the device status word;
 * the launch then drains).  The objective F(x_k) of every problem runs as a
 * second persistent launch.  Supported: ZERO / SYM / PER wavelet boundaries
 * with every level longer than 2L' (not PPD), PSF radius <= 12.
 *
 * adjwt_fista_batch_workspace_size: device bytes for the count problems (u
 * and g images, LL buffers, momentum and objective partials of each).
 * adjwt_fista_batch_create: probs / x / y are HOST arrays of count entries;
 * x[i], y[i] the DEVICE coefficient vectors of problem i (its state, as in
 * adjwt_fista_state); ws: the workspace, 256-byte aligned, which the batch
 * uses until destroyed.  The plans, observations and state buffers must
 * outlive the batch.  Creation uploads the item tables (allocates device
 * memory once); later calls allocate nothing.  Errors: INVALID_ARG, SHAPE
 * (an unsupported problem), ALIGN, WORKSPACE, CUDA.
 * adjwt_fista_batch_reset: t_1 = 1 for every problem (the caller zeroes or
 * sets x and y, with y = x).  adjwt_fista_batch_set_iteration: the momentum
 * every problem has after k iterations from t_1 = 1 (to continue the runs of
 * a rebuilt batch whose problems kept their x and y); 0 <= k <= 1e8.
 * adjwt_fista_batch_run: iters iterations of every problem, one launch
 * (plus a memset of its counters) on `stream`.
 * adjwt_fista_batch_objective: objectives_dev[i] (DEVICE doubles) =
 * F(x_i) = 1/2 ||R W x_i - b_i||^2 + lambda_i ||x_i||_1, one launch.
 * adjwt_fista_batch_wait_selftest: one launch in which the first item waits
 * for a stage that never runs: after about a second it records
 * ADJWT_ERR_TIMEOUT in the device status word and the launch drains (a
 * test of the bounded waits; the other problems may have advanced, so reset
 * the batch before using it again).
 * adjwt_fista_batch_info: items per iteration, stages, resident CTAs.
 * The launches of one batch share its counters and workspace: issue them on
 * one stream (or otherwise serialise them). */
typedef struct adjwt_fista_batch adjwt_fista_batch;
size_t adjwt_fista_batch_workspace_size(int count, const adjwt_fista_problem* probs);
int adjwt_fista_batch_create(adjwt_fista_batch** out, int count, const adjwt_fista_problem* probs, float* const* x,
                             float* const* y, void* ws, size_t ws_bytes);
void adjwt_fista_batch_destroy(adjwt_fista_batch* batch);
int adjwt_fista_batch_reset(const adjwt_fista_batch* batch, adjwt_stream_t stream);
int adjwt_fista_batch_set_iteration(const adjwt_fista_batch* batch, int64_t k, adjwt_stream_t stream);
int adjwt_fista_batch_run(const adjwt_fista_batch* batch, int iters, adjwt_stream_t stream);
int adjwt_fista_batch_objective(const adjwt_fista_batch* batch, double* objectives_dev, adjwt_stream_t stream);
int adjwt_fista_batch_wait_selftest(const adjwt_fista_batch* batch, adjwt_stream_t stream);
int adjwt_fista_batch_info(const adjwt_fista_batch* batch, int* items_per_iteration, int* stages, int* ctas);

/* FISTA's momentum as fista_step applies it (HOST, no device work):
 * t_next = (1 + sqrt(1 + 4 t^2))/2 and beta = (t - 1)/t_next rounded to
 * float32, the weight of y_{k+1} = x_k + beta (x_k - x_{k-1}).  t >= 1 and
 * finite, pointers non-NULL (INVALID_ARG). */
int adjwt_fista_momentum(double t, double* t_next, float* beta);

/* The same iteration with the momentum t_k resident in the workspace (no
 * counterpart in the paper: it makes an iteration a pure sequence of stream
 * operations that can be captured in a CUDA graph and replayed, e.g. to run
 * many independent problems concurrently).  x (x_{k-1} -> x_k) and y
 * (y_k -> y_{k+1}) are device coefficient vectors; the workspace holds t_k,
 * which adjwt_fista_device_reset sets to 1 (start of a solve) and every call
 * advances.  If objective_dev (DEVICE double, 8-byte aligned) is non-NULL it
 * receives F(x_k).  Nothing synchronises.  Errors as fista_step, plus ALIAS
 * when the workspace overlaps x or y. */
int fista_step_device(const adjwt_fista_problem* prob, float* x, float* y, void* ws, size_t ws_bytes,
                      double* objective_dev, adjwt_stream_t stream);
int adjwt_fista_device_reset(const adjwt_fista_problem* prob, void* ws, size_t ws_bytes, adjwt_stream_t stream);

/* F(x) = 1/2 ||R W x - b||^2 + lambda ||x||_1 into *objective_out (HOST);
 * synchronises the stream. */
int adjwt_fista_objective(const adjwt_fista_problem* prob, const float* x, void* ws, size_t ws_bytes,
                          double* objective_out, adjwt_stream_t stream);

/* Step size: power iteration on A^*A, A = R W.  v (device coeffs) holds the
 * start vector and receives the last normalised iterate; after `iters` steps
 * *lipschitz_out (HOST) = 1.01 * ||A^*A v_{iters-1}|| with ||v|| = 1.
 * Synchronises the stream. */
int adjwt_fista_lipschitz(const adjwt_fista_problem* prob, float* v, int iters, void* ws, size_t ws_bytes,
                          double* lipschitz_out, adjwt_stream_t stream);

/* ------------------------------------------------------ differentiation
 * Pieces for differentiating through the FISTA iteration (unrolled FISTA;
 * gradients with respect to lambda, the PSF width sigma and the data b).
 * The backward of x_{k+1} = S_tau(y_k - (1/L) A^*(A y_k - b)), A = R W
 * (Sec. 1, Eq. 1), applies A and A^* themselves (the chain rule
 * A^* grad l(A x) of Sec. 1, correct only with the exact adjoint) plus the
 * elementwise steps below.  None has a counterpart in the paper beyond that.
 *
 * adjwt_gaussian_taps (HOST): taps[i] = e_i / sum_j e_j,
 * e_i = exp(-(i - (k-1)/2)^2 / (2 sigma^2)), and, if dtaps_dsigma is not
 * NULL, its derivative dtaps[i] = taps[i] (d_i^2 - sum_j taps[j] d_j^2) /
 * sigma^3 (host arrays of k doubles).  For the separable PSF g (x) g,
 * dR/dsigma = R[g', g] + R[g, g'] (two blur plans).  SHAPE unless k is odd
 * and >= 1; INVALID_ARG unless sigma > 0.
 *
 * adjwt_axpby: out[i] = a x[i] + b y[i], i < n (device float32; out may
 * alias x or y).
 *
 * adjwt_soft_threshold: out[i] = sign(in[i]) max(|in[i]| - tau, 0), i < n,
 * the soft threshold of the FISTA prox (Sec. I-B) on its own (e.g. to
 * sparsify a warm start); out may alias in; tau >= 0 finite (INVALID_ARG).
 *
 * adjwt_dot: *out_dev (DEVICE double) = sum over rows x cols of x y, both
 * arrays with row pitch `pitch` floats (a coefficient vector: rows = 1,
 * cols = pitch = length).  Float64 per-block partials, added in a fixed
 * order (reproducible).  ws: device scratch of adjwt_reduce_workspace_size()
 * bytes (WORKSPACE if smaller or NULL).
 *
 * fista_prox_vjp: vector-Jacobian product of the soft threshold
 * x_{k+1} = S_tau(z): zbar[i] = xbar[i] if x_next[i] != 0 else 0 (S_tau(z) is
 * zero exactly where |z| <= tau), and *sign_dot_dev (DEVICE double) =
 * sum_i sign(x_next[i]) xbar[i], so that dl/dtau = -(*sign_dot_dev).  zbar
 * may alias xbar.  ws as for adjwt_dot. */
int adjwt_gaussian_taps(int k, double sigma, double* taps, double* dtaps_dsigma);
size_t adjwt_reduce_workspace_size(void);
int adjwt_axpby(int64_t n, float a, const float* x, float b, const float* y, float* out, adjwt_stream_t stream);
int adjwt_soft_threshold(int64_t n, const float* in, double tau, float* out, adjwt_stream_t stream);
int adjwt_dot(int rows, int64_t cols, int64_t pitch, const float* x, const float* y, double* out_dev, void* ws,
              size_t ws_bytes, adjwt_stream_t stream);
int fista_prox_vjp(int64_t n, const float* x_next, const float* xbar, float* zbar, double* sign_dot_dev, void* ws,
                   size_t ws_bytes, adjwt_stream_t stream);

/* One whole reverse-mode step of the FISTA iteration k (0-based) for the
 * exact-adjoint problem (prob->gradient == ADJWT_GRAD_ADJOINT, else
 * INVALID_ARG): the kernels of the pieces above, W, R, R^* and W^* issued in
 * one call.  With beta = beta_k (the momentum factor that iteration used, as
 * float32), x_next = x_{k+1}, y_k (device coefficient vectors), xbar = the
 * adjoint of x_{k+1} collected so far and ybar = the adjoint of y_{k+1}:
 *   X = xbar + (1 + beta) ybar;  zbar = X where x_next != 0;  u = W zbar
 *   *dtau_dev -= sum sign(x_next) X                       (tau = lambda / L)
 *   ybar <- zbar - (1/L) W^* R^* R u     (the adjoint of y_k)
 *   xbar <- -beta (old ybar)              (the adjoint of x_k from y_{k+1})
 *   db   += (1/L) R u                     (if db, a device image, is not NULL)
 *   *dsigma_dev -= (1/L) (<R' u, R W y_k - b> + <R u, R' W y_k>)
 * where R' = dblur_1 + dblur_2, the two plans of dR/dsigma
 * (adjwt_gaussian_taps).  dsigma_dev NULL skips that term (and the plans may
 * be NULL); otherwise both plans are required (INVALID_ARG) and describe the
 * problem's image (SHAPE).  dtau_dev and dsigma_dev are DEVICE doubles that
 * the call accumulates into (float64).  Vectors 16-byte aligned (ALIGN).
 * ws: device scratch of adjwt_fista_vjp_workspace_size(prob) bytes, 256-byte
 * aligned (WORKSPACE), overlapping none of the arguments.  Nothing
 * synchronises; the call is a pure sequence of stream operations. */
size_t adjwt_fista_vjp_workspace_size(const adjwt_fista_problem* prob);
int fista_vjp_step(const adjwt_fista_problem* prob, const adjwt_blur_plan* dblur_1, const adjwt_blur_plan* dblur_2,
                   const float* x_next, const float* y_k, double beta, float* xbar, float* ybar, float* db,
                   double* dtau_dev, double* dsigma_dev, void* ws, size_t ws_bytes, adjwt_stream_t stream);

/* Measured float32 FMA rate of the current device in TFLOP/s (no
 * counterpart in the paper; it gives the blur and channel-gradient rooflines
 * their float32 ceiling): independent FMA chains on every SM, no memory
 * traffic, best of five timed launches.  Synchronises the stream; allocates
 * nothing.  INVALID_ARG (NULL), CUDA. */
int adjwt_fp32_fma_peak(double* tflops, adjwt_stream_t stream);

/* ------------------------------------------------------------------- tracing
 * Optional per-kernel device timing without a profiler (the paper has no
 * counterpart; it serves the measurement harness).  adjwt_trace_enable(n)
 * arms a pool of n CUDA event pairs: each kernel launched afterwards by this
 * library (from one host thread) is bracketed by two events on its stream
 * until the pool is full; adjwt_trace_enable(0) disarms and frees the pool.
 * adjwt_trace_reset() reuses the pool from record 0.  adjwt_trace_get waits
 * for record i and returns the kernel's name (static string), its tag (the
 * wavelet level, else 0) and its duration in milliseconds. */
int adjwt_trace_enable(int capacity);
int adjwt_trace_reset(void);
int adjwt_trace_count(void);
int adjwt_trace_get(int i, const char** name, int* tag, float* ms);
/* Device milliseconds from the start of trace record `first` to the end of
 * record `last` (first <= last, same stream): one multi-kernel call, launch
 * gaps included.  INVALID_ARG for indices outside the records. */
int adjwt_trace_span(int first, int last, float* ms);
/* What the armed pool records: level 1 (the default) every kernel; level 2
 * only whole operator calls, one record each, named "op:wt_synth" (W),
 * "op:blur_normal" (R^*(R u - b)), "op:wt_adjoint_prox" (W^* with the FISTA
 * prox, or W^dagger for the variant), "op:momentum" (fista_step_device) and
 * "op:conv_gradient".  No events then sit between the kernels of one
 * operator, so programmatic dependent launch overlaps them as it does
 * untraced.  INVALID_ARG for other levels. */
int adjwt_trace_set_level(int level);

#ifdef __cplusplus
}
#endif
#endif /* ADJWT_H */
