// One reverse-mode step of unrolled FISTA (the solve of Eq. 1) as a single
// call: the same kernels a caller would chain (W, R, R^*, W^*, the soft
// threshold's vector-Jacobian product, a x + b y, inner products), issued
// from here so that a backward pass costs one host call per iteration.
//
// Iteration k (0-based): z_k = y_k - (1/L) A^*(A y_k - b), A = R W,
// x_{k+1} = soft(z_k, lambda/L), y_{k+1} = x_{k+1} + beta_k (x_{k+1} - x_k).
// Given Xp (adjoint of x_{k+1} collected so far) and Y (adjoint of y_{k+1}):
//   X = Xp + (1 + beta_k) Y;  zbar = X [x_{k+1} != 0];  dtau -= sum sign(x_{k+1}) X
//   u = W zbar;  Y <- zbar - (1/L) W^* R^* R u;  Xp <- -beta_k Y_{k+1};  db += (1/L) R u
//   dsigma -= (1/L) (<R' u, R W y_k - b> + <R u, R' W y_k>),  R' = R[g', g] + R[g, g'].
// The chain rule A^* grad l(A x) of Sec. I needs the exact adjoint W^* (Eq. 4).
#include <cstdint>

#include "adjwt_internal.h"

namespace adjwt {
namespace {

struct VjpWs {
  float *ll0, *ll1;
  float *u, *Ru, *t1, *Wy, *r, *t2, *t3;  // images (rows x image_pitch)
  float *X, *zbar, *q;                    // coefficient vectors
  double *pa, *pb;                        // partial sums
  size_t bytes;
};

VjpWs layout_vjp(const adjwt_wt_plan* wt, char* base) {
  VjpWs w{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += static_cast<size_t>(round_up(static_cast<int64_t>(bytes), 256));
    return p;
  };
  const size_t img = static_cast<size_t>(wt->rows) * wt->image_pitch * sizeof(float);
  const size_t cof = static_cast<size_t>(wt->num_coeffs) * sizeof(float);
  w.ll0 = reinterpret_cast<float*>(take(static_cast<size_t>(wt->ll_buf_floats[0]) * 4));
  w.ll1 = reinterpret_cast<float*>(take(static_cast<size_t>(wt->ll_buf_floats[1]) * 4));
  float** imgs[] = {&w.u, &w.Ru, &w.t1, &w.Wy, &w.r, &w.t2, &w.t3};
  for (float** p : imgs) *p = reinterpret_cast<float*>(take(img));
  float** cofs[] = {&w.X, &w.zbar, &w.q};
  for (float** p : cofs) *p = reinterpret_cast<float*>(take(cof));
  w.pa = reinterpret_cast<double*>(take(reduce_partials_bytes()));
  w.pb = reinterpret_cast<double*>(take(reduce_partials_bytes()));
  w.bytes = off;
  return w;
}

}  // namespace
}  // namespace adjwt

using namespace adjwt;

extern "C" size_t adjwt_fista_vjp_workspace_size(const adjwt_fista_problem* prob) {
  if (!prob || !prob->wt) return 0;
  return layout_vjp(prob->wt, nullptr).bytes;
}

extern "C" int fista_vjp_step(const adjwt_fista_problem* prob, const adjwt_blur_plan* dblur_1,
                              const adjwt_blur_plan* dblur_2, const float* x_next, const float* y_k, double beta,
                              float* xbar, float* ybar, float* db, double* dtau_dev, double* dsigma_dev, void* ws,
                              size_t ws_bytes, adjwt_stream_t stream) {
  if (!prob || !prob->wt || !prob->blur || !prob->b)
    return fail(ADJWT_ERR_INVALID_ARG, "fista_vjp_step: problem, plans or b missing");
  if (!(prob->lipschitz > 0.0)) return fail(ADJWT_ERR_INVALID_ARG, "fista_vjp_step: lipschitz must be > 0");
  if (prob->gradient != ADJWT_GRAD_ADJOINT)
    return fail(ADJWT_ERR_INVALID_ARG, "fista_vjp_step: only the exact-adjoint gradient is differentiable");
  const bool want_sigma = dsigma_dev != nullptr;
  if (want_sigma && (!dblur_1 || !dblur_2))
    return fail(ADJWT_ERR_INVALID_ARG, "fista_vjp_step: dsigma needs both derivative blur plans");
  if (!x_next || !y_k || !xbar || !ybar || !dtau_dev)
    return fail(ADJWT_ERR_INVALID_ARG, "fista_vjp_step: NULL vector or accumulator");
  for (const void* v : {static_cast<const void*>(x_next), static_cast<const void*>(y_k),
                        static_cast<const void*>(xbar), static_cast<const void*>(ybar), static_cast<const void*>(db)})
    if (reinterpret_cast<uintptr_t>(v) & 15u) return fail(ADJWT_ERR_ALIGN, "fista_vjp_step: vector not 16-byte aligned");
  const size_t need = adjwt_fista_vjp_workspace_size(prob);
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < need)
    return fail(ADJWT_ERR_WORKSPACE, "fista_vjp_step: workspace of adjwt_fista_vjp_workspace_size bytes, "
                                     "256-byte aligned, needed");
  const adjwt_wt_plan* wt = prob->wt;
  const adjwt_blur_plan* R = prob->blur;
  if (R->rows != wt->rows || R->cols != wt->cols || R->image_pitch != wt->image_pitch)
    return fail(ADJWT_ERR_SHAPE, "fista_vjp_step: wavelet and blur plans describe different images");
  if (want_sigma && (dblur_1->rows != wt->rows || dblur_1->cols != wt->cols || dblur_2->rows != wt->rows ||
                     dblur_2->cols != wt->cols))
    return fail(ADJWT_ERR_SHAPE, "fista_vjp_step: derivative blur plans describe a different image");
  int rc = ADJWT_OK;
  const VjpWs w = layout_vjp(wt, static_cast<char*>(ws));
  cudaStream_t s = stream;
  const int rows = wt->rows;
  const int64_t cols = wt->cols, pitch = wt->image_pitch, nc = wt->num_coeffs;
  const float il = static_cast<float>(1.0 / prob->lipschitz);
  const float fb = static_cast<float>(beta);
  ProxArgs none{};
  int np = 0;
  // X = Xp + (1 + beta) Y;  zbar, dtau
  rc = launch_axpby(1, nc, nc, 1.0f, xbar, 1.0f + fb, ybar, w.X, s);
  if (!rc) rc = launch_prox_vjp_partials(nc, x_next, w.X, w.zbar, w.pa, s, &np);
  if (!rc) rc = launch_sum_partials(w.pa, np, -1.0, dtau_dev, 1, 1.0, dtau_dev, s);
  // u = W zbar, Ru = R u, q = W^* R^* R u
  if (!rc) rc = launch_wt_synth(wt, w.zbar, w.u, w.ll0, w.ll1, s);
  if (!rc) rc = launch_blur(R, w.u, w.Ru, false, s);
  if (!rc) rc = launch_blur(R, w.Ru, w.t1, true, s);
  if (!rc) rc = launch_wt_analysis(wt, w.t1, w.q, true, none, w.ll0, w.ll1, s, nullptr);
  // Xp <- -beta Y_{k+1}, then Y <- zbar - (1/L) q
  if (!rc) rc = launch_axpby(1, nc, nc, -fb, ybar, 0.0f, ybar, xbar, s);
  if (!rc) rc = launch_axpby(1, nc, nc, 1.0f, w.zbar, -il, w.q, ybar, s);
  if (!rc && db) rc = launch_axpby(rows, cols, pitch, 1.0f, db, il, w.Ru, db, s);
  if (rc || !want_sigma) return rc;
  // dsigma -= (1/L) (<R' u, R W y_k - b> + <R u, R' W y_k>)
  rc = launch_wt_synth(wt, y_k, w.Wy, w.ll0, w.ll1, s);
  if (!rc) rc = launch_blur(R, w.Wy, w.t1, false, s);
  if (!rc) rc = launch_axpby(rows, cols, pitch, 1.0f, w.t1, -1.0f, prob->b, w.r, s);
  if (!rc) rc = launch_blur(dblur_1, w.u, w.t2, false, s);
  if (!rc) rc = launch_blur(dblur_2, w.u, w.t3, false, s);
  if (!rc) rc = launch_axpby(rows, cols, pitch, 1.0f, w.t2, 1.0f, w.t3, w.t2, s);
  if (!rc) rc = launch_dot_partials(rows, cols, pitch, w.t2, w.r, w.pa, s, &np);
  if (!rc) rc = launch_sum_partials(w.pa, np, -1.0 / prob->lipschitz, dsigma_dev, 1, 1.0, dsigma_dev, s);
  if (!rc) rc = launch_blur(dblur_1, w.Wy, w.t3, false, s);
  if (!rc) rc = launch_blur(dblur_2, w.Wy, w.t1, false, s);
  if (!rc) rc = launch_axpby(rows, cols, pitch, 1.0f, w.t3, 1.0f, w.t1, w.t3, s);
  if (!rc) rc = launch_dot_partials(rows, cols, pitch, w.Ru, w.t3, w.pb, s, &np);
  if (!rc) rc = launch_sum_partials(w.pb, np, -1.0 / prob->lipschitz, dsigma_dev, 1, 1.0, dsigma_dev, s);
  return rc;
}
