"""Learned warm start for the solve of Eq. 1 (argument marshalling only).

FISTA as the paper runs it (Sec. I-B) starts from zero.  Here a network of
eight 3x3 convolution layers (1 -> 32, six 32 -> 32, 32 -> 1, ReLU, residual
output u_hat = b + net(b)) estimates the image from the observation b, and
FISTA starts from x_0 = W^dagger u_hat.  Every step runs in libadjwt's
kernels behind include/adjwt_cnn.h: the forward and the data gradient of the
32 -> 32 layers on tcgen05, their weight gradient on the warp MMA, the thin
layers, the loss and Adam on the CUDA cores.  This module allocates the
buffers with torch and passes pointers.

Images are (n, rows, pitch) float32 tensors (the (rows, image_pitch) layout
of the transform and blur plans, stacked); hidden activations are bf16
(n, rows, cols, 32).
"""
import ctypes as C

import torch

from . import _lib, _ptr, _stream, lib, soft_threshold, workspace, wt_analysis


# (Cout, Cin) of the eight 3x3 layers
LAYER_SHAPES = [(32, 1)] + [(32, 32)] * 6 + [(1, 32)]


def param_count():
    return int(lib().adjwt_cnn_param_count())


def _f32(t, numel, name):
    if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or t.numel() < numel:
        raise ValueError(f"{name}: need a contiguous float32 CUDA tensor with >= {numel} elements")


class WarmStartNet:
    """Parameters (flat float32, layer by layer: weights (Cout, Cin, 3, 3),
    then biases), their packed bf16 tensor-core operands and the Adam state."""

    def __init__(self, params):
        n = param_count()
        self.params = torch.as_tensor(params, dtype=torch.float32).to("cuda").contiguous()
        if self.params.numel() != n:
            raise ValueError(f"need {n} parameters")
        self.grad = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step_count = 0
        self.packed = workspace(lib().adjwt_cnn_packed_bytes())
        self.loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        self._act = {}
        self._ws = {}
        self.pack()

    def pack(self, stream=None):
        _lib.check(lib().cnn_pack(_ptr(self.params), _ptr(self.packed), _stream(stream)))

    def _buffers(self, n, rows, cols):
        key = (n, rows, cols)
        if key not in self._act:
            self._act[key] = workspace(lib().adjwt_cnn_activation_bytes(n, rows, cols))
            self._ws[key] = workspace(lib().adjwt_cnn_workspace_size(n, rows, cols))
        return self._act[key], self._ws[key]

    def forward(self, b, rows, cols, u_hat=None, stream=None):
        """u_hat (n, rows, pitch) for observations b of the same layout."""
        n, pitch = b.shape[0], b.shape[-1]
        _f32(b, n * rows * pitch, "b")
        u_hat = torch.empty_like(b) if u_hat is None else u_hat
        _f32(u_hat, n * rows * pitch, "u_hat")
        act, _ = self._buffers(n, rows, cols)
        _lib.check(lib().cnn_forward(n, rows, cols, _ptr(b), pitch, _ptr(self.params), _ptr(self.packed), _ptr(act),
                                     _ptr(u_hat), _stream(stream)))
        return u_hat

    def backward(self, b, u_hat, u_ref, rows, cols, stream=None):
        """self.grad = d loss / d params and self.loss (device float64) =
        1/(2 n rows cols) sum (u_hat - u_ref)^2, after forward(b)."""
        n, pitch = b.shape[0], b.shape[-1]
        for t, name in ((b, "b"), (u_hat, "u_hat"), (u_ref, "u_ref")):
            _f32(t, n * rows * pitch, name)
        act, ws = self._buffers(n, rows, cols)
        _lib.check(lib().cnn_backward(n, rows, cols, _ptr(b), _ptr(u_hat), _ptr(u_ref), pitch, _ptr(self.params),
                                      _ptr(self.packed), _ptr(act), _ptr(self.grad), _ptr(self.loss), _ptr(ws),
                                      ws.numel(), _stream(stream)))
        return self.grad

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        self.step_count += 1
        _lib.check(lib().cnn_adam(self.params.numel(), _ptr(self.params), _ptr(self.grad), _ptr(self.m),
                                  _ptr(self.v), self.step_count, float(lr), float(beta1), float(beta2), float(eps),
                                  _stream(stream)))
        self.pack(stream)

    def train_step(self, b, u_ref, rows, cols, lr=1e-3, stream=None):
        """One forward, backward and Adam step; returns the device loss."""
        u_hat = self.forward(b, rows, cols, stream=stream)
        self.backward(b, u_hat, u_ref, rows, cols, stream=stream)
        self.adam(lr, stream=stream)
        return self.loss

    def warm_start(self, wt, b, tau=0.0, stream=None):
        """x_0 = S_tau(W^dagger u_hat) for one observation b ((rows, image_pitch)
        image of plan wt); tau > 0 soft-thresholds the analysis coefficients
        (tau = lambda / L_f is the threshold of one FISTA prox)."""
        u_hat = self.forward(b.reshape(1, wt.rows, wt.image_pitch), wt.rows, wt.cols, stream=stream)
        x0 = wt_analysis(wt, u_hat.reshape(wt.rows, wt.image_pitch), stream=stream)
        return soft_threshold(x0, tau, out=x0, stream=stream) if tau > 0 else x0


def conv32(n, rows, cols, x, packed_layer, bias=None, relu=False, mask=None, out=None, stream=None):
    """One 32 -> 32 layer on the tensor cores; x, mask, out: (n, rows, cols, 32) bf16."""
    out = torch.empty_like(x) if out is None else out
    _lib.check(lib().cnn_conv32(n, rows, cols, _ptr(x), _ptr(packed_layer), _ptr(bias), 1 if relu else 0,
                                _ptr(mask), _ptr(out), _stream(stream)))
    return out


def conv32_wgrad(n, rows, cols, x, dz, stream=None):
    """(grad_w (32, 32, 3, 3), grad_b (32,)) of a 32 -> 32 layer."""
    gw = torch.empty(32 * 32 * 9, dtype=torch.float32, device=x.device)
    gb = torch.empty(32, dtype=torch.float32, device=x.device)
    ws = workspace(lib().adjwt_cnn_wgrad_workspace_size(), device=x.device)
    _lib.check(lib().cnn_conv32_wgrad(n, rows, cols, _ptr(x), _ptr(dz), _ptr(gw), _ptr(gb), _ptr(ws), ws.numel(),
                                      _stream(stream)))
    return gw.reshape(32, 32, 3, 3), gb


def packed_layer(net, layer, direction=0):
    """The packed operand block of 32 -> 32 layer `layer` (1..6): direction 0
    forward, 1 data gradient."""
    block = 18432
    off = ((layer - 1) * 2 + direction) * block
    return net.packed[off:off + block]


def _main():
    """Train the network for a few steps on seeded blurred images
    (python -m paper_1707_02018_gb300.warmstart --batch 8 --size 512 --steps 5):
    observations R u + noise of piecewise-smooth images u (9 x 9 Gaussian,
    sigma 1.5, symmetric boundary), targets u.  Prints the losses."""
    import argparse

    from synthetic_inputs import gaussian_noise, he_normal_params, piecewise_smooth_image

    from . import BlurPlan, blur, gaussian_taps

    ap = argparse.ArgumentParser()
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--lr", type=float, default=1e-3)
    args = ap.parse_args()
    n, size = args.batch, args.size
    g, _ = gaussian_taps(9, 1.5)
    bl = BlurPlan(size, size, g, g, "sym")
    pitch = bl.image_pitch
    b = torch.zeros(n, size, pitch, dtype=torch.float32, device="cuda")
    u = torch.zeros_like(b)
    for i in range(n):
        u[i, :, :size] = torch.as_tensor(piecewise_smooth_image(size, size, 500 + i), dtype=torch.float32)
        blur(bl, u[i], out=b[i])
        b[i, :, :size] += torch.as_tensor(gaussian_noise((size, size), 600 + i, 1e-3), dtype=torch.float32,
                                          device="cuda")
    net = WarmStartNet(he_normal_params(LAYER_SHAPES, 700))
    losses = [float(net.train_step(b, u, size, size, lr=args.lr)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    print("losses", " ".join(f"{v:.4e}" for v in losses))


if __name__ == "__main__":
    _main()
