// FISTA for the synthesis-formulation deblurring problem (Eq. 1):
//   min_x 1/2 ||R W x - b||^2 + lambda ||x||_1,  grad f(x) = W^* R^* (R W x - b).
// One iteration is three stream-ordered stages: W (per-level reconstruction
// kernels), the fused R^*(R u - b) kernel, and W^* whose per-level kernels
// apply the proximal step and the momentum update in their epilogue, so the
// gradient never reaches HBM.  Reductions (objective, norms) accumulate in
// float64 per CTA and are summed by one CTA in a fixed order.
#include <algorithm>
#include <cmath>

#include "adjwt_internal.h"
#include "device_common.cuh"

namespace adjwt {
namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_sum_partials(const double* a, int na, double sa, const double* b,
                                                           int nb, double sb, double* out) {
  pdl_entry();
  __shared__ double red[kThreads / 32];
  double ta = 0.0, tb = 0.0;
  for (int i = threadIdx.x; i < na; i += kThreads) ta += a[i];
  for (int i = threadIdx.x; i < nb; i += kThreads) tb += b[i];
  const double va = block_sum<kThreads>(ta, red);
  __syncthreads();
  const double vb = block_sum<kThreads>(tb, red);
  if (threadIdx.x == 0) out[0] = sa * va + sb * vb;
}

__global__ void __launch_bounds__(kThreads) k_sq_norm(const float* v, int64_t count, double* partials, int absval) {
  pdl_entry();
  __shared__ double red[kThreads / 32];
  float acc = 0.0f;  // per-thread float32 partial, float64 across the block and the grid
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < count; i += (int64_t)gridDim.x * kThreads) {
    const float x = v[i];
    acc = absval ? acc + fabsf(x) : fmaf(x, x, acc);
  }
  const double t = block_sum<kThreads>((double)acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void k_scale(float* v, int64_t count, const double* sq_norm) {
  pdl_entry();
  const float s = static_cast<float>(1.0 / sqrt(sq_norm[0]));
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    v[i] *= s;
}

// Device-resident momentum: m[0] = t_k; one thread advances it and stores
// m[1] = (t_k - 1)/t_{k+1} for the prox epilogues of the same iteration.
__global__ void k_momentum(double* m) {
  pdl_entry();
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const double t = m[0];
    // rounded like the host's 0.5 * (1 + sqrt(1 + 4 t t)): no fused multiply-add
    const double t1 = 0.5 * (1.0 + sqrt(__dadd_rn(1.0, __dmul_rn(4.0 * t, t))));
    m[1] = (t - 1.0) / t1;
    m[0] = t1;
  }
}

__global__ void k_momentum_reset(double* m) {
  pdl_entry();
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    m[0] = 1.0;
    m[1] = 0.0;
  }
}

constexpr int kNormBlocks = 304;  // 2 x 152 SMs

struct FistaWs {
  float* ll0;
  float* ll1;
  float* u;
  float* g;
  float* bv;  // blur scratch image (R u - b)
  double* part_a;
  double* part_b;
  double* scalars;  // [0] result, [1] scratch
  double* momentum; // [0] t_k, [1] beta (device-resident momentum)
  size_t bytes;
};

FistaWs layout_ws(const adjwt_fista_problem* pr, char* base) {
  const adjwt_wt_plan* w = pr->wt;
  FistaWs L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += static_cast<size_t>(round_up(static_cast<int64_t>(bytes), 256));
    return p;
  };
  const size_t img = static_cast<size_t>(w->rows) * w->image_pitch * sizeof(float);
  L.ll0 = reinterpret_cast<float*>(take(w->ll_buf_floats[0] * sizeof(float)));
  L.ll1 = reinterpret_cast<float*>(take(w->ll_buf_floats[1] * sizeof(float)));
  L.u = reinterpret_cast<float*>(take(img));
  L.g = reinterpret_cast<float*>(take(img));
  L.bv = reinterpret_cast<float*>(take(img));
  const int slots = std::max(std::max(wt_l1_partial_slots(w), blur_partial_slots(pr->blur)), kNormBlocks);
  L.part_a = reinterpret_cast<double*>(take(slots * sizeof(double)));
  L.part_b = reinterpret_cast<double*>(take(slots * sizeof(double)));
  L.scalars = reinterpret_cast<double*>(take(4 * sizeof(double)));
  L.momentum = reinterpret_cast<double*>(take(2 * sizeof(double)));
  L.bytes = off;
  return L;
}

int finish_scalar(double* dev, double* host, cudaStream_t s) {
  ADJWT_CUDA_CHECK(cudaMemcpyAsync(host, dev, sizeof(double), cudaMemcpyDeviceToHost, s));
  ADJWT_CUDA_CHECK(cudaStreamSynchronize(s));
  if (!std::isfinite(*host)) return fail(ADJWT_ERR_NONFINITE, "objective or norm is not finite");
  return ADJWT_OK;
}

// F(x) into *out (device; ws.scalars by default), using ws.u and the partial buffers.
int objective_async(const adjwt_fista_problem* pr, const float* x, const FistaWs& W, bool have_l1, int l1_slots,
                    cudaStream_t s, double* out = nullptr) {
  if (!out) out = W.scalars;
  int rc = launch_wt_synth(pr->wt, x, W.u, W.ll0, W.ll1, s);
  if (rc) return rc;
  int nb = 0;
  rc = launch_blur_residual_norm(pr->blur, W.u, pr->b, W.part_b, s, &nb);
  if (rc) return rc;
  if (!have_l1) {
    ADJWT_TRACED("l1_norm", 0, s, pdl_launch(k_sq_norm, kNormBlocks, kThreads, 0, s, x, pr->wt->num_coeffs, W.part_a, 1));
    ADJWT_CUDA_CHECK(cudaGetLastError());
    l1_slots = kNormBlocks;
  }
  ADJWT_TRACED("sum_partials", 0, s,
               pdl_launch(k_sum_partials, 1, kThreads, 0, s, W.part_a, l1_slots, pr->lambda, W.part_b, nb, 1.0, out));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  return ADJWT_OK;
}

}  // namespace

int launch_sum_partials(const double* a, int na, double sa, const double* b, int nb, double sb, double* out,
                        cudaStream_t s) {
  ADJWT_TRACED("sum_partials", 0, s, pdl_launch(k_sum_partials, 1, kThreads, 0, s, a, na, sa, b, nb, sb, out));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  return ADJWT_OK;
}

size_t fista_workspace_bytes(const adjwt_fista_problem* pr) { return layout_ws(pr, nullptr).bytes; }

// FISTA's momentum (the method cited in Sec. I-B): t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2
// and the extrapolation weight beta_k = (t_k - 1)/t_{k+1}, rounded to float32
// as the prox epilogue applies it.
void fista_momentum(double t, double* t_next, float* beta) {
  const double t1 = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
  *t_next = t1;
  *beta = static_cast<float>((t - 1.0) / t1);
}

int fista_step_impl(const adjwt_fista_problem* pr, adjwt_fista_state* st, void* ws, double* objective_out,
                    cudaStream_t s) {
  const FistaWs W = layout_ws(pr, static_cast<char*>(ws));
  int rc = 0;
  ADJWT_TRACED_OP("op:wt_synth", 0, s, rc = launch_wt_synth(pr->wt, st->y, W.u, W.ll0, W.ll1, s));
  if (rc) return rc;
  ADJWT_TRACED_OP("op:blur_normal", 0, s, rc = launch_blur_normal(pr->blur, W.u, pr->b, W.g, nullptr, W.bv, s, nullptr));
  if (rc) return rc;
  double t1 = 0.0;
  float beta = 0.0f;
  fista_momentum(st->t, &t1, &beta);
  ProxArgs prox{};
  prox.x = st->x;
  prox.y = st->y;
  prox.step = static_cast<float>(1.0 / pr->lipschitz);
  prox.thresh = static_cast<float>(pr->lambda / pr->lipschitz);
  prox.beta = beta;
  prox.l1_partials = objective_out ? W.part_a : nullptr;
  int l1_slots = 0;
  ADJWT_TRACED_OP("op:wt_adjoint_prox", 0, s,
                  rc = launch_wt_analysis(pr->wt, W.g, nullptr, pr->gradient == ADJWT_GRAD_ADJOINT, prox, W.ll0,
                                          W.ll1, s, &l1_slots));
  if (rc) return rc;
  st->t = t1;
  st->k += 1;
  if (objective_out) {
    rc = objective_async(pr, st->x, W, true, l1_slots, s);
    if (rc) return rc;
    return finish_scalar(W.scalars, objective_out, s);
  }
  return ADJWT_OK;
}

// One iteration with the momentum t_k kept in the workspace: no host state and
// no synchronisation, so a sequence of iterations can be captured in a CUDA
// graph and replayed.  With objective_dev (device) non-null, F(x_k) is
// written there.
int fista_step_device_impl(const adjwt_fista_problem* pr, float* x, float* y, void* ws, double* objective_dev,
                           cudaStream_t s) {
  const FistaWs W = layout_ws(pr, static_cast<char*>(ws));
  cudaError_t me = cudaSuccess;
  ADJWT_TRACED_OP("op:momentum", 0, s,
                  ADJWT_TRACED("momentum", 0, s, me = pdl_launch(k_momentum, 1, 32, 0, s, W.momentum)));
  ADJWT_CUDA_CHECK(me);
  ADJWT_CUDA_CHECK(cudaGetLastError());
  int rc = 0;
  ADJWT_TRACED_OP("op:wt_synth", 0, s, rc = launch_wt_synth(pr->wt, y, W.u, W.ll0, W.ll1, s));
  if (rc) return rc;
  ADJWT_TRACED_OP("op:blur_normal", 0, s, rc = launch_blur_normal(pr->blur, W.u, pr->b, W.g, nullptr, W.bv, s, nullptr));
  if (rc) return rc;
  ProxArgs prox{};
  prox.x = x;
  prox.y = y;
  prox.step = static_cast<float>(1.0 / pr->lipschitz);
  prox.thresh = static_cast<float>(pr->lambda / pr->lipschitz);
  prox.beta_dev = W.momentum + 1;
  prox.l1_partials = objective_dev ? W.part_a : nullptr;
  int l1_slots = 0;
  ADJWT_TRACED_OP("op:wt_adjoint_prox", 0, s,
                  rc = launch_wt_analysis(pr->wt, W.g, nullptr, pr->gradient == ADJWT_GRAD_ADJOINT, prox, W.ll0,
                                          W.ll1, s, &l1_slots));
  if (rc) return rc;
  if (objective_dev) return objective_async(pr, x, W, true, l1_slots, s, objective_dev);
  return ADJWT_OK;
}

int fista_device_reset_impl(const adjwt_fista_problem* pr, void* ws, cudaStream_t s) {
  const FistaWs W = layout_ws(pr, static_cast<char*>(ws));
  ADJWT_TRACED("momentum", 0, s, pdl_launch(k_momentum_reset, 1, 32, 0, s, W.momentum));
  ADJWT_CUDA_CHECK(cudaGetLastError());
  return ADJWT_OK;
}

int fista_objective_impl(const adjwt_fista_problem* pr, const float* x, void* ws, double* out, cudaStream_t s) {
  const FistaWs W = layout_ws(pr, static_cast<char*>(ws));
  int rc = objective_async(pr, x, W, false, 0, s);
  if (rc) return rc;
  return finish_scalar(W.scalars, out, s);
}

int fista_lipschitz_impl(const adjwt_fista_problem* pr, float* v, int iters, void* ws, double* out, cudaStream_t s) {
  const FistaWs W = layout_ws(pr, static_cast<char*>(ws));
  const int64_t C = pr->wt->num_coeffs;
  auto normalise = [&]() -> int {
    ADJWT_TRACED("sq_norm", 0, s, pdl_launch(k_sq_norm, kNormBlocks, kThreads, 0, s, v, C, W.part_a, 0));
    ADJWT_TRACED("sum_partials", 0, s,
                 pdl_launch(k_sum_partials, 1, kThreads, 0, s, W.part_a, kNormBlocks, 1.0, nullptr, 0, 0.0, W.scalars));
    ADJWT_TRACED("scale", 0, s, pdl_launch(k_scale, kNormBlocks, kThreads, 0, s, v, C, W.scalars));
    ADJWT_CUDA_CHECK(cudaGetLastError());
    return ADJWT_OK;
  };
  int rc = normalise();
  if (rc) return rc;
  ProxArgs none{};
  for (int it = 0; it < iters; ++it) {
    rc = launch_wt_synth(pr->wt, v, W.u, W.ll0, W.ll1, s);
    if (rc) return rc;
    rc = launch_blur_normal(pr->blur, W.u, nullptr, W.g, nullptr, W.bv, s, nullptr);
    if (rc) return rc;
    rc = launch_wt_analysis(pr->wt, W.g, v, true, none, W.ll0, W.ll1, s, nullptr);
    if (rc) return rc;
    rc = normalise();  // scalars[0] = ||A^*A v||^2 of this step
    if (rc) return rc;
  }
  double sq = 0.0;
  rc = finish_scalar(W.scalars, &sq, s);
  if (rc) return rc;
  if (!(sq > 0.0)) return fail(ADJWT_ERR_NONFINITE, "power iteration collapsed to zero");
  *out = 1.01 * std::sqrt(sq);
  return ADJWT_OK;
}

}  // namespace adjwt
