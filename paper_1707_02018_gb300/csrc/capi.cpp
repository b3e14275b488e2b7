// extern "C" entry points of libadjwt: argument validation, workspace
// carving, and dispatch to the stream-ordered launchers.  Nothing here throws;
// every failure returns an ADJWT_ERR_* code and records a message.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>

#include "adjwt_internal.h"

namespace adjwt {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return ADJWT_ERR_CUDA;
}

size_t fista_workspace_bytes(const adjwt_fista_problem* pr);
int fista_step_impl(const adjwt_fista_problem* pr, adjwt_fista_state* st, void* ws, double* objective_out,
                    cudaStream_t s);
int fista_objective_impl(const adjwt_fista_problem* pr, const float* x, void* ws, double* out, cudaStream_t s);
int fista_step_device_impl(const adjwt_fista_problem* pr, float* x, float* y, void* ws, double* objective_dev,
                           cudaStream_t s);
int fista_device_reset_impl(const adjwt_fista_problem* pr, void* ws, cudaStream_t s);
int fista_lipschitz_impl(const adjwt_fista_problem* pr, float* v, int iters, void* ws, double* out,
                         cudaStream_t s);

namespace {

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + nb && y < x + na;
}

int check_ptr(const void* p, const char* name) {
  if (!p) return fail(ADJWT_ERR_INVALID_ARG, std::string(name) + " is NULL");
  if (!aligned16(p)) return fail(ADJWT_ERR_ALIGN, std::string(name) + " is not 16-byte aligned");
  return ADJWT_OK;
}

int check_ws(const void* ws, size_t have, size_t need, const char* who) {
  if (need == 0) return ADJWT_OK;
  if (!ws) return fail(ADJWT_ERR_WORKSPACE, std::string(who) + ": workspace is NULL");
  if ((reinterpret_cast<uintptr_t>(ws) & 255u) != 0)
    return fail(ADJWT_ERR_WORKSPACE, std::string(who) + ": workspace not 256-byte aligned");
  if (have < need)
    return fail(ADJWT_ERR_WORKSPACE, std::string(who) + ": workspace of " + std::to_string(have) +
                                         " bytes, need " + std::to_string(need));
  return ADJWT_OK;
}

size_t image_bytes(int rows, int pitch) { return static_cast<size_t>(rows) * pitch * sizeof(float); }

void split_wt_ws(const adjwt_wt_plan* p, void* ws, float** b0, float** b1) {
  char* base = static_cast<char*>(ws);
  *b0 = reinterpret_cast<float*>(base);
  *b1 = reinterpret_cast<float*>(base + round_up(p->ll_buf_floats[0] * 4, 256));
}

int wt_common(const adjwt_wt_plan* p, const float* in, size_t in_bytes, const float* out, size_t out_bytes,
              void* ws, size_t ws_bytes, const char* who) {
  if (!p) return fail(ADJWT_ERR_INVALID_ARG, std::string(who) + ": plan is NULL");
  int rc = check_ptr(in, "input");
  if (!rc) rc = check_ptr(out, "output");
  if (rc) return rc;
  if (overlap(in, in_bytes, out, out_bytes)) return fail(ADJWT_ERR_ALIAS, std::string(who) + ": output overlaps input");
  rc = check_ws(ws, ws_bytes, adjwt_wt_workspace_size(p), who);
  if (rc) return rc;
  if (ws && (overlap(ws, adjwt_wt_workspace_size(p), in, in_bytes) ||
             overlap(ws, adjwt_wt_workspace_size(p), out, out_bytes)))
    return fail(ADJWT_ERR_ALIAS, std::string(who) + ": workspace overlaps a tensor");
  return ADJWT_OK;
}

int check_problem(const adjwt_fista_problem* pr) {
  if (!pr || !pr->wt || !pr->blur) return fail(ADJWT_ERR_INVALID_ARG, "fista: problem or plan is NULL");
  if (pr->wt->rows != pr->blur->rows || pr->wt->cols != pr->blur->cols)
    return fail(ADJWT_ERR_SHAPE, "fista: wavelet and blur plans describe different images");
  if (!(pr->lambda >= 0.0) || !std::isfinite(pr->lambda)) return fail(ADJWT_ERR_INVALID_ARG, "fista: bad lambda");
  if (!(pr->lipschitz > 0.0) || !std::isfinite(pr->lipschitz))
    return fail(ADJWT_ERR_INVALID_ARG, "fista: lipschitz must be finite and > 0");
  if (pr->gradient != ADJWT_GRAD_ADJOINT && pr->gradient != ADJWT_GRAD_PINV)
    return fail(ADJWT_ERR_INVALID_ARG, "fista: unknown gradient mode");
  return check_ptr(pr->b, "b");
}

}  // namespace
}  // namespace adjwt

using namespace adjwt;

extern "C" const char* adjwt_last_error(void) { return g_last_error.c_str(); }
extern "C" int adjwt_version(void) { return 1; }

extern "C" int wt_synth(const adjwt_wt_plan* p, const float* coeffs, float* image, void* ws, size_t ws_bytes,
                        adjwt_stream_t stream) {
  if (!p) return fail(ADJWT_ERR_INVALID_ARG, "wt_synth: plan is NULL");
  int rc = wt_common(p, coeffs, p->num_coeffs * 4, image, image_bytes(p->rows, p->image_pitch), ws, ws_bytes,
                     "wt_synth");
  if (rc) return rc;
  float *b0, *b1;
  split_wt_ws(p, ws, &b0, &b1);
  return launch_wt_synth(p, coeffs, image, b0, b1, stream);
}

static int analysis_entry(const adjwt_wt_plan* p, const float* image, float* coeffs, void* ws, size_t ws_bytes,
                          adjwt_stream_t stream, bool adjoint, const char* who) {
  if (!p) return fail(ADJWT_ERR_INVALID_ARG, std::string(who) + ": plan is NULL");
  int rc = wt_common(p, image, image_bytes(p->rows, p->image_pitch), coeffs, p->num_coeffs * 4, ws, ws_bytes, who);
  if (rc) return rc;
  float *b0, *b1;
  split_wt_ws(p, ws, &b0, &b1);
  ProxArgs none{};
  return launch_wt_analysis(p, image, coeffs, adjoint, none, b0, b1, stream, nullptr);
}

extern "C" int wt_synth_adjoint(const adjwt_wt_plan* p, const float* image, float* coeffs, void* ws,
                                size_t ws_bytes, adjwt_stream_t stream) {
  return analysis_entry(p, image, coeffs, ws, ws_bytes, stream, true, "wt_synth_adjoint");
}

extern "C" int wt_analysis(const adjwt_wt_plan* p, const float* image, float* coeffs, void* ws, size_t ws_bytes,
                           adjwt_stream_t stream) {
  return analysis_entry(p, image, coeffs, ws, ws_bytes, stream, false, "wt_analysis");
}

static int blur_entry(const adjwt_blur_plan* p, const float* in, float* out, adjwt_stream_t stream, bool adjoint) {
  if (!p) return fail(ADJWT_ERR_INVALID_ARG, "blur: plan is NULL");
  int rc = check_ptr(in, "input");
  if (!rc) rc = check_ptr(out, "output");
  if (rc) return rc;
  const size_t nb = image_bytes(p->rows, p->image_pitch);
  if (overlap(in, nb, out, nb)) return fail(ADJWT_ERR_ALIAS, "blur: output overlaps input");
  return launch_blur(p, in, out, adjoint, stream);
}

extern "C" int blur(const adjwt_blur_plan* p, const float* in, float* out, adjwt_stream_t stream) {
  return blur_entry(p, in, out, stream, false);
}

extern "C" int blur_adjoint(const adjwt_blur_plan* p, const float* in, float* out, adjwt_stream_t stream) {
  return blur_entry(p, in, out, stream, true);
}

extern "C" int blur_normal(const adjwt_blur_plan* p, const float* u, const float* b, float* g, double* half_sq_out,
                           void* ws, size_t ws_bytes, adjwt_stream_t stream) {
  if (!p) return fail(ADJWT_ERR_INVALID_ARG, "blur_normal: plan is NULL");
  int rc = check_ptr(u, "u");
  if (!rc) rc = check_ptr(g, "g");
  if (!rc && b) rc = check_ptr(b, "b");
  if (rc) return rc;
  const size_t nb = image_bytes(p->rows, p->image_pitch);
  if (overlap(u, nb, g, nb) || (b && overlap(b, nb, g, nb)))
    return fail(ADJWT_ERR_ALIAS, "blur_normal: g overlaps an input");
  double* parts = nullptr;
  float* v = nullptr;
  if (half_sq_out || ws) {
    rc = check_ws(ws, ws_bytes, adjwt_blur_workspace_size(p), "blur_normal");
    if (rc) return rc;
    if (overlap(ws, adjwt_blur_workspace_size(p), u, nb) || overlap(ws, adjwt_blur_workspace_size(p), g, nb) ||
        (b && overlap(ws, adjwt_blur_workspace_size(p), b, nb)))
      return fail(ADJWT_ERR_ALIAS, "blur_normal: workspace overlaps a tensor");
    parts = half_sq_out ? static_cast<double*>(ws) : nullptr;
    v = reinterpret_cast<float*>(static_cast<char*>(ws) + blur_partials_bytes(p));
  }
  int np = 0;
  rc = launch_blur_normal(p, u, b, g, parts, v, stream, &np);
  if (rc) return rc;
  if (half_sq_out) return launch_sum_partials(parts, np, 1.0, nullptr, 0, 0.0, half_sq_out, stream);
  return ADJWT_OK;
}

extern "C" size_t adjwt_conv_adjoint_workspace_size(int batch, int64_t n, int k) {
  if (batch <= 0 || n <= 0 || k <= 0) return 0;
  return static_cast<size_t>(round_up(conv_partial_floats(batch, n, k) * 4, 256));
}

extern "C" int conv_adjoint(int batch, int64_t n, int k, const float* s, const float* h, const float* r,
                            float* grad_h, float* grad_s, void* ws, size_t ws_bytes, adjwt_stream_t stream) {
  if (batch < 0 || n < 1 || k < 1) return fail(ADJWT_ERR_SHAPE, "conv_adjoint: need batch >= 0, n >= 1, k >= 1");
  if (batch > 65535) return fail(ADJWT_ERR_SHAPE, "conv_adjoint: batch above 65535");
  if (batch == 0 || (!grad_h && !grad_s)) return ADJWT_OK;
  int rc = check_ptr(r, "r");
  if (!rc && grad_h) rc = check_ptr(s, "s");
  if (!rc && grad_s) rc = check_ptr(h, "h");
  if (!rc && grad_h) rc = check_ptr(grad_h, "grad_h");
  if (!rc && grad_s) rc = check_ptr(grad_s, "grad_s");
  if (rc) return rc;
  const size_t sb = (size_t)batch * n * 4, hb = (size_t)batch * k * 4, rb = (size_t)batch * (n + k - 1) * 4;
  if (grad_h && (overlap(grad_h, hb, s, sb) || overlap(grad_h, hb, r, rb) || (h && overlap(grad_h, hb, h, hb))))
    return fail(ADJWT_ERR_ALIAS, "conv_adjoint: grad_h overlaps an input");
  if (grad_s && (overlap(grad_s, sb, r, rb) || overlap(grad_s, sb, h, hb) || (s && overlap(grad_s, sb, s, sb))))
    return fail(ADJWT_ERR_ALIAS, "conv_adjoint: grad_s overlaps an input");
  if (grad_h) {
    rc = check_ws(ws, ws_bytes, adjwt_conv_adjoint_workspace_size(batch, n, k), "conv_adjoint");
    if (rc) return rc;
  }
  return launch_conv_adjoint(batch, n, k, s, h, r, grad_h, grad_s, static_cast<float*>(ws), stream);
}

extern "C" int conv_adjoint_noalloc(int batch, int64_t n, int k, const float* s, const float* h, const float* r,
                                    float* grad_h, float* grad_s, adjwt_stream_t stream) {
  if (batch < 0 || n < 1 || k < 1)
    return fail(ADJWT_ERR_SHAPE, "conv_adjoint_noalloc: need batch >= 0, n >= 1, k >= 1");
  if (batch > 65535) return fail(ADJWT_ERR_SHAPE, "conv_adjoint_noalloc: batch above 65535");
  if (batch == 0 || (!grad_h && !grad_s)) return ADJWT_OK;
  if (grad_h && conv_partial_floats(batch, n, k) > conv_static_scratch_floats())
    return fail(ADJWT_ERR_WORKSPACE,
                "conv_adjoint_noalloc: grad_h needs batch * ceil(n / c) * k = " +
                    std::to_string(conv_partial_floats(batch, n, k)) +
                    " partial sums (c = the kernel's chunk: 16 * floor((4097 - 16 * ceil(k / 16)) / 16) for k <= 1024, "
                    "1024 above), more than the fixed scratch of " + std::to_string(conv_static_scratch_floats()) +
                    " floats; use conv_adjoint with a workspace");
  int rc = check_ptr(r, "r");
  if (!rc && grad_h) rc = check_ptr(s, "s");
  if (!rc && grad_s) rc = check_ptr(h, "h");
  if (!rc && grad_h) rc = check_ptr(grad_h, "grad_h");
  if (!rc && grad_s) rc = check_ptr(grad_s, "grad_s");
  if (rc) return rc;
  const size_t sb = (size_t)batch * n * 4, hb = (size_t)batch * k * 4, rb = (size_t)batch * (n + k - 1) * 4;
  if (grad_h && (overlap(grad_h, hb, s, sb) || overlap(grad_h, hb, r, rb) || (h && overlap(grad_h, hb, h, hb))))
    return fail(ADJWT_ERR_ALIAS, "conv_adjoint_noalloc: grad_h overlaps an input");
  if (grad_s && (overlap(grad_s, sb, r, rb) || overlap(grad_s, sb, h, hb) || (s && overlap(grad_s, sb, s, sb))))
    return fail(ADJWT_ERR_ALIAS, "conv_adjoint_noalloc: grad_s overlaps an input");
  return launch_conv_adjoint_noalloc(batch, n, k, s, h, r, grad_h, grad_s, stream);
}

// Eq. 6 workspace: the replicated source and the per-channel source
// gradients (C x n floats each), then the channel-gradient workspace.
extern "C" size_t adjwt_bce_gradient_workspace_size(int channels, int64_t n, int k) {
  if (channels <= 0 || n <= 0 || k <= 0) return 0;
  const size_t rows = static_cast<size_t>(round_up((int64_t)channels * n * 4, 256));
  return 2 * rows + adjwt_conv_gradient_workspace_size(channels, n, k);
}

extern "C" int bce_gradient(int channels, int64_t n, int k, const float* s, const float* h, const float* x,
                            double lambda_tv, double delta, float* grad_h, float* grad_s, void* ws, size_t ws_bytes,
                            adjwt_stream_t stream) {
  if (channels < 1 || n < 1 || k < 1) return fail(ADJWT_ERR_SHAPE, "bce_gradient: need channels, n, k >= 1");
  if (channels > 65535 || k > 4096) return fail(ADJWT_ERR_SHAPE, "bce_gradient: channels above 65535 or k above 4096");
  if (!(delta > 0.0) || !std::isfinite(delta) || !(lambda_tv >= 0.0) || !std::isfinite(lambda_tv))
    return fail(ADJWT_ERR_INVALID_ARG, "bce_gradient: need delta > 0 and lambda_tv >= 0, finite");
  int rc = check_ptr(s, "s");
  if (!rc) rc = check_ptr(h, "h");
  if (!rc) rc = check_ptr(x, "x");
  if (!rc && grad_h) rc = check_ptr(grad_h, "grad_h");
  if (!rc && grad_s) rc = check_ptr(grad_s, "grad_s");
  if (rc) return rc;
  const size_t sb = (size_t)n * 4, hb = (size_t)channels * k * 4, xb = (size_t)channels * (n + k - 1) * 4;
  const void* ins[3] = {s, h, x};
  const size_t inb[3] = {sb, hb, xb};
  for (int i = 0; i < 3; ++i) {
    if (grad_h && overlap(grad_h, hb, ins[i], inb[i])) return fail(ADJWT_ERR_ALIAS, "bce_gradient: grad_h overlaps an input");
    if (grad_s && overlap(grad_s, sb, ins[i], inb[i])) return fail(ADJWT_ERR_ALIAS, "bce_gradient: grad_s overlaps an input");
  }
  if (grad_h && grad_s && overlap(grad_h, hb, grad_s, sb)) return fail(ADJWT_ERR_ALIAS, "bce_gradient: outputs overlap");
  const size_t need = adjwt_bce_gradient_workspace_size(channels, n, k);
  rc = check_ws(ws, ws_bytes, need, "bce_gradient");
  if (rc) return rc;
  if (!grad_h && !grad_s) return ADJWT_OK;
  const size_t rows = static_cast<size_t>(round_up((int64_t)channels * n * 4, 256));
  float* s_rows = static_cast<float*>(ws);
  float* gs_rows = reinterpret_cast<float*>(static_cast<char*>(ws) + rows);
  void* cws = static_cast<char*>(ws) + 2 * rows;
  for (int c = 0; c < channels; ++c)
    ADJWT_CUDA_CHECK(cudaMemcpyAsync(s_rows + (size_t)c * n, s, sb, cudaMemcpyDeviceToDevice, stream));
  rc = conv_gradient(channels, n, k, s_rows, h, x, nullptr, grad_h, grad_s ? gs_rows : nullptr, cws,
                     adjwt_conv_gradient_workspace_size(channels, n, k), stream);
  if (rc) return rc;
  return launch_bce_finish(channels, n, k, h, grad_h, gs_rows, grad_s, lambda_tv, delta, stream);
}

extern "C" size_t adjwt_conv_gradient_workspace_size(int batch, int64_t n, int k) {
  if (batch <= 0 || n <= 0 || k <= 0) return 0;
  size_t bytes = adjwt_conv_adjoint_workspace_size(batch, n, k);
  if (!conv_fused_supported(k)) bytes += static_cast<size_t>(round_up((int64_t)batch * (n + k - 1) * 4, 256));
  return bytes;
}

extern "C" int conv_gradient(int batch, int64_t n, int k, const float* s, const float* h, const float* x, float* r,
                             float* grad_h, float* grad_s, void* ws, size_t ws_bytes, adjwt_stream_t stream) {
  if (batch < 0 || n < 1 || k < 1) return fail(ADJWT_ERR_SHAPE, "conv_gradient: need batch >= 0, n >= 1, k >= 1");
  if (batch > 65535) return fail(ADJWT_ERR_SHAPE, "conv_gradient: batch above 65535");
  if (k > 4096) return fail(ADJWT_ERR_SHAPE, "conv_gradient: k above 4096");
  if (batch == 0) return ADJWT_OK;
  int rc = check_ptr(s, "s");
  if (!rc) rc = check_ptr(h, "h");
  if (!rc && x) rc = check_ptr(x, "x");
  if (!rc && r) rc = check_ptr(r, "r");
  if (!rc && grad_h) rc = check_ptr(grad_h, "grad_h");
  if (!rc && grad_s) rc = check_ptr(grad_s, "grad_s");
  if (rc) return rc;
  const size_t sb = (size_t)batch * n * 4, hb = (size_t)batch * k * 4, rb = (size_t)batch * (n + k - 1) * 4;
  const void* ins[3] = {s, h, x};
  const size_t inb[3] = {sb, hb, rb};
  void* outs[3] = {r, grad_h, grad_s};
  const size_t outb[3] = {rb, hb, sb};
  for (int o = 0; o < 3; ++o) {
    if (!outs[o]) continue;
    for (int i = 0; i < 3; ++i)
      if (ins[i] && overlap(outs[o], outb[o], ins[i], inb[i]))
        return fail(ADJWT_ERR_ALIAS, "conv_gradient: an output overlaps an input");
    for (int p = o + 1; p < 3; ++p)
      if (outs[p] && overlap(outs[o], outb[o], outs[p], outb[p]))
        return fail(ADJWT_ERR_ALIAS, "conv_gradient: outputs overlap");
  }
  const size_t need = adjwt_conv_gradient_workspace_size(batch, n, k);
  rc = check_ws(ws, ws_bytes, need, "conv_gradient");
  if (rc) return rc;
  float* partials = static_cast<float*>(ws);
  if (conv_fused_supported(k)) {
    ADJWT_TRACED_OP("op:conv_gradient", 0, stream,
                    rc = launch_conv_fused(batch, n, k, s, h, x, nullptr, r, grad_h, grad_s, partials, stream));
    return rc;
  }
  // long channels: residual into r (or the workspace), then the adjoint
  float* rbuf = r ? r : reinterpret_cast<float*>(static_cast<char*>(ws) + adjwt_conv_adjoint_workspace_size(batch, n, k));
  rc = launch_conv_residual(batch, n, k, h, s, x, rbuf, stream);
  if (rc) return rc;
  if (!grad_h && !grad_s) return ADJWT_OK;
  return launch_conv_adjoint(batch, n, k, s, h, rbuf, grad_h, grad_s, partials, stream);
}

extern "C" int conv_residual(int batch, int64_t n, int k, const float* h, const float* s, const float* x, float* r,
                             adjwt_stream_t stream) {
  if (batch < 0 || n < 1 || k < 1) return fail(ADJWT_ERR_SHAPE, "conv_residual: need batch >= 0, n >= 1, k >= 1");
  if (batch > 65535) return fail(ADJWT_ERR_SHAPE, "conv_residual: batch above 65535");
  if (batch == 0) return ADJWT_OK;
  int rc = check_ptr(h, "h");
  if (!rc) rc = check_ptr(s, "s");
  if (!rc) rc = check_ptr(r, "r");
  if (!rc && x) rc = check_ptr(x, "x");
  if (rc) return rc;
  const size_t rb = (size_t)batch * (n + k - 1) * 4;
  if (overlap(r, rb, h, (size_t)batch * k * 4) || overlap(r, rb, s, (size_t)batch * n * 4))
    return fail(ADJWT_ERR_ALIAS, "conv_residual: r overlaps an input");
  return launch_conv_residual(batch, n, k, h, s, x, r, stream);
}

extern "C" size_t adjwt_fista_workspace_size(const adjwt_fista_problem* pr) {
  if (!pr || !pr->wt || !pr->blur) return 0;
  return fista_workspace_bytes(pr);
}

extern "C" int fista_step_device(const adjwt_fista_problem* pr, float* x, float* y, void* ws, size_t ws_bytes,
                                 double* objective_dev, adjwt_stream_t stream) {
  int rc = check_problem(pr);
  if (rc) return rc;
  rc = check_ptr(x, "x");
  if (!rc) rc = check_ptr(y, "y");
  if (rc) return rc;
  if (objective_dev && (reinterpret_cast<uintptr_t>(objective_dev) & 7u))
    return fail(ADJWT_ERR_ALIGN, "fista_step_device: objective_dev is not 8-byte aligned");
  const size_t cb = pr->wt->num_coeffs * 4;
  if (overlap(x, cb, y, cb)) return fail(ADJWT_ERR_ALIAS, "fista_step_device: x and y overlap");
  rc = check_ws(ws, ws_bytes, fista_workspace_bytes(pr), "fista_step_device");
  if (rc) return rc;
  const size_t wb = fista_workspace_bytes(pr);
  if (overlap(ws, wb, x, cb) || overlap(ws, wb, y, cb))
    return fail(ADJWT_ERR_ALIAS, "fista_step_device: workspace overlaps the state");
  return fista_step_device_impl(pr, x, y, ws, objective_dev, stream);
}

extern "C" int adjwt_fista_device_reset(const adjwt_fista_problem* pr, void* ws, size_t ws_bytes,
                                        adjwt_stream_t stream) {
  int rc = check_problem(pr);
  if (rc) return rc;
  rc = check_ws(ws, ws_bytes, fista_workspace_bytes(pr), "adjwt_fista_device_reset");
  if (rc) return rc;
  return fista_device_reset_impl(pr, ws, stream);
}

extern "C" int fista_step(const adjwt_fista_problem* pr, adjwt_fista_state* st, void* ws, size_t ws_bytes,
                          double* objective_out, adjwt_stream_t stream) {
  int rc = check_problem(pr);
  if (rc) return rc;
  if (!st) return fail(ADJWT_ERR_INVALID_ARG, "fista_step: state is NULL");
  rc = check_ptr(st->x, "x");
  if (!rc) rc = check_ptr(st->y, "y");
  if (rc) return rc;
  if (!(st->t >= 1.0) || !std::isfinite(st->t)) return fail(ADJWT_ERR_INVALID_ARG, "fista_step: t must be >= 1");
  const size_t cb = pr->wt->num_coeffs * 4;
  if (overlap(st->x, cb, st->y, cb)) return fail(ADJWT_ERR_ALIAS, "fista_step: x and y overlap");
  rc = check_ws(ws, ws_bytes, fista_workspace_bytes(pr), "fista_step");
  if (rc) return rc;
  return fista_step_impl(pr, st, ws, objective_out, stream);
}

extern "C" int adjwt_fista_objective(const adjwt_fista_problem* pr, const float* x, void* ws, size_t ws_bytes,
                                     double* objective_out, adjwt_stream_t stream) {
  int rc = check_problem(pr);
  if (rc) return rc;
  rc = check_ptr(x, "x");
  if (rc) return rc;
  if (!objective_out) return fail(ADJWT_ERR_INVALID_ARG, "objective_out is NULL");
  rc = check_ws(ws, ws_bytes, fista_workspace_bytes(pr), "fista_objective");
  if (rc) return rc;
  return fista_objective_impl(pr, x, ws, objective_out, stream);
}

extern "C" int adjwt_fista_lipschitz(const adjwt_fista_problem* pr, float* v, int iters, void* ws, size_t ws_bytes,
                                     double* lipschitz_out, adjwt_stream_t stream) {
  if (!pr || !pr->wt || !pr->blur) return fail(ADJWT_ERR_INVALID_ARG, "fista_lipschitz: problem or plan is NULL");
  if (pr->wt->rows != pr->blur->rows || pr->wt->cols != pr->blur->cols)
    return fail(ADJWT_ERR_SHAPE, "fista_lipschitz: plans describe different images");
  int rc = check_ptr(v, "v");
  if (rc) return rc;
  if (iters < 1) return fail(ADJWT_ERR_INVALID_ARG, "fista_lipschitz: iters must be >= 1");
  if (!lipschitz_out) return fail(ADJWT_ERR_INVALID_ARG, "lipschitz_out is NULL");
  rc = check_ws(ws, ws_bytes, fista_workspace_bytes(pr), "fista_lipschitz");
  if (rc) return rc;
  return fista_lipschitz_impl(pr, v, iters, ws, lipschitz_out, stream);
}

extern "C" int adjwt_fista_momentum(double t, double* t_next, float* beta) {
  if (!t_next || !beta) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_fista_momentum: t_next and beta must be non-NULL");
  if (!(t >= 1.0) || !std::isfinite(t)) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_fista_momentum: need finite t >= 1");
  fista_momentum(t, t_next, beta);
  return ADJWT_OK;
}
