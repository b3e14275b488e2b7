/* Learned warm start for the solve of Eq. 1 (C ABI of libadjwt).
 *
 * FISTA as the paper runs it (Sec. I-B) starts from x_0 = 0.  A learned warm
 * start computes an image estimate u_hat from the observation b with a small
 * convolutional network and starts FISTA from x_0 = W^dagger u_hat (the
 * coefficient vector of the redundant transform is not image-shaped, so the
 * network predicts the image).  The paper has no network; this one is:
 *
 *   a_0 = b (1 channel);  a_l = relu(conv3x3(a_{l-1}; w_l, c_l)), l = 1..7 (32 channels)
 *   u_hat = b + conv3x3(a_7; w_8, c_8)
 *
 * conv3x3: 'same' cross-correlation with zero padding,
 *   y[n, i, j, o] = c[o] + sum_{ci, dy, dx} w[o, ci, dy, dx] x[n, i+dy-1, j+dx-1, ci].
 * Training loss l = 1/(2 n rows cols) sum (u_hat - u_ref)^2, optimiser Adam.
 *
 * Conventions (in addition to those of adjwt.h):
 *  - Parameters: one float32 DEVICE vector of adjwt_cnn_param_count()
 *    (56,097) values, layer by layer: the weights in (Cout, Cin, 3, 3) order,
 *    then the Cout biases (layers: 1->32, six 32->32, 32->1).
 *  - Single-channel images (b, u_hat, u_ref): float32 DEVICE, n images of
 *    rows x cols with row pitch `pitch` floats (>= cols), images stacked.
 *  - Hidden activations and their gradients: bfloat16 DEVICE, channels last,
 *    (n, rows, cols, 32) dense (64 bytes a pixel).  The activation buffer
 *    holds a_1 .. a_7 one after another (adjwt_cnn_activation_bytes).
 *  - Arithmetic: the 32 -> 32 layers multiply bfloat16 operands (the weights
 *    rounded to bfloat16 by cnn_pack) with float32 accumulation on the
 *    tensor cores; the 1 -> 32 and 32 -> 1 layers use float32 weights.
 *  - Pointers 16-byte aligned (ALIGN); sizes >= 0 (SHAPE); an empty batch
 *    does nothing.  Nothing synchronises the stream; every call is a pure
 *    sequence of kernel launches that can be captured in a CUDA graph. */
#ifndef ADJWT_CNN_H
#define ADJWT_CNN_H

#include "adjwt.h"

#ifdef __cplusplus
extern "C" {
#endif

size_t adjwt_cnn_param_count(void);
/* Bytes of the packed bf16 tensor-core operands (cnn_pack). */
size_t adjwt_cnn_packed_bytes(void);
/* Bytes of the activation buffer a_1 .. a_7 for n images of rows x cols. */
size_t adjwt_cnn_activation_bytes(int n, int rows, int cols);
/* Bytes of the cnn_backward workspace (256-byte aligned). */
size_t adjwt_cnn_workspace_size(int n, int rows, int cols);

/* Pack the weights of the six 32 -> 32 layers into the bf16 operand layout
 * of the tensor-core kernels: for layer l (1..6), a forward block then a
 * data-gradient block (taps flipped, channels swapped) of 18,432 bytes each.
 * Call after every change of params. */
int cnn_pack(const float* params, void* packed, adjwt_stream_t stream);

/* u_hat for n observations b; act (adjwt_cnn_activation_bytes) receives
 * a_1 .. a_7 for cnn_backward. */
int cnn_forward(int n, int rows, int cols, const float* b, int64_t pitch, const float* params, const void* packed,
                void* act, float* u_hat, adjwt_stream_t stream);

/* grad (param-count floats, overwritten) = d l / d params at the point of the
 * preceding cnn_forward (same b, params, packed and act; u_hat its output),
 * and *loss_dev (DEVICE double) = l.  Hidden-activation gradients are stored
 * in bfloat16.  ws: adjwt_cnn_workspace_size(n, rows, cols) bytes. */
int cnn_backward(int n, int rows, int cols, const float* b, const float* u_hat, const float* u_ref, int64_t pitch,
                 const float* params, const void* packed, const void* act, float* grad, double* loss_dev, void* ws,
                 size_t ws_bytes, adjwt_stream_t stream);

/* One Adam step (Kingma & Ba) of step number `step` >= 1 on `count` values:
 *   m = beta1 m + (1-beta1) g;  v = beta2 v + (1-beta2) g^2;
 *   params -= lr (m / (1-beta1^step)) / (sqrt(v / (1-beta2^step)) + eps).
 * m and v: float32 DEVICE state, zero before step 1.  INVALID_ARG unless
 * 0 <= beta < 1, eps > 0, lr >= 0 and step >= 1. */
int cnn_adam(int64_t count, float* params, const float* grad, float* m, float* v, int64_t step, double lr,
             double beta1, double beta2, double eps, adjwt_stream_t stream);

/* One 32 -> 32 layer on the tensor cores (the pieces cnn_forward and
 * cnn_backward use):
 *   out[p][o] = mask(p, o) * act(c[o] + sum_{tap, ci} B[tap][o][ci] in[p + offset_tap][ci])
 * with B the packed block packed_layer (a forward block: the layer itself; a
 * data-gradient block: its adjoint), bias c (NULL: none), act = relu if relu
 * else identity, mask(p, o) = [mask[p][o] > 0] if mask is not NULL else 1.
 * in, mask, out: (n, rows, cols, 32) bf16; out may not overlap in (ALIAS). */
int cnn_conv32(int n, int rows, int cols, const void* in, const void* packed_layer, const float* bias, int relu,
               const void* mask, void* out, adjwt_stream_t stream);

/* Weight and bias gradient of a 32 -> 32 layer with input x and output
 * gradient dz (both (n, rows, cols, 32) bf16):
 *   grad_w[o][ci][dy][dx] = sum_p dz[p][o] x[p + (dy-1, dx-1)][ci]  (zero outside)
 *   grad_b[o] = sum_p dz[p][o]
 * (float32 DEVICE, overwritten; warp-level bf16 MMAs, float32 per-CTA
 * partials summed in float64 in a fixed order).  ws:
 * adjwt_cnn_wgrad_workspace_size() bytes. */
size_t adjwt_cnn_wgrad_workspace_size(void);
int cnn_conv32_wgrad(int n, int rows, int cols, const void* x, const void* dz, float* grad_w, float* grad_b, void* ws,
                     size_t ws_bytes, adjwt_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* ADJWT_CNN_H */
