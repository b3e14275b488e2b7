"""FP64 oracle of the learned warm start for the solve of Eq. 1.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper solves Eq. 1 with FISTA from a zero start (Sec. I-B); a learned
warm start replaces that start with x_0 = W^dagger u_hat, where u_hat is an
image estimate computed from the observation b by a small convolutional
network (the paper has no network; its definition here is a reading):

  a_0 = b                                   (one channel)
  a_l = relu(conv3x3(a_{l-1}; w_l, c_l))    l = 1 .. 7, 32 channels
  u_hat = b + conv3x3(a_7; w_8, c_8)        (one channel, residual output)

conv3x3 is the 'same' cross-correlation with zero padding,
  y[n, i, j, o] = c[o] + sum_{ci, dy, dx} w[o, ci, dy, dx] x[n, i+dy-1, j+dx-1, ci],
on channels-last arrays (n, rows, cols, channels).  The training loss is
l = 1/(2 n rows cols) sum (u_hat - u_ref)^2, minimised by Adam.

``bf16=True`` emulates the storage precision of the GPU path: the weights of
the 32 -> 32 layers and the hidden activations (and their gradients) are
rounded to bfloat16 (round to nearest even of their float32 value); the
arithmetic itself stays float64.
"""
import numpy as np

HIDDEN = 32
LAYERS = 8


# ------------------------------------------------------------------ bfloat16
def round_bf16(a):
    """Round to the nearest bfloat16 (ties to even), through float32: the
    value a float32 accumulator holds, then its top 16 bits rounded."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = ((u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


# --------------------------------------------------------------- conv3x3
def conv3x3(x, w, c=None):
    """'Same' 3x3 cross-correlation with zero padding; x (n, H, W, Cin),
    w (Cout, Cin, 3, 3), c (Cout,) or None -> (n, H, W, Cout)."""
    x = np.asarray(x, dtype=np.float64)
    n, H, W, _ = x.shape
    xp = np.zeros((n, H + 2, W + 2, x.shape[3]))
    xp[:, 1:H + 1, 1:W + 1] = x
    y = np.zeros((n, H, W, w.shape[0]))
    for dy in range(3):
        for dx in range(3):
            y += xp[:, dy:dy + H, dx:dx + W, :] @ np.asarray(w[:, :, dy, dx], dtype=np.float64).T
    if c is not None:
        y += np.asarray(c, dtype=np.float64)
    return y


def conv3x3_backward(x, w, dy):
    """Gradients of sum(dy * conv3x3(x, w, c)) with respect to x, w and c:
      dx[n, i, j, ci] = sum_{o, dy, dx} w[o, ci, dy, dx] dy[n, i-dy+1, j-dx+1, o]
      dw[o, ci, dy, dx] = sum_{n, i, j} dy[n, i, j, o] x[n, i+dy-1, j+dx-1, ci]
      dc[o] = sum_{n, i, j} dy[n, i, j, o]."""
    x = np.asarray(x, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    n, H, W, _ = x.shape
    xp = np.zeros((n, H + 2, W + 2, x.shape[3]))
    xp[:, 1:H + 1, 1:W + 1] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros(w.shape)
    for ky in range(3):
        for kx in range(3):
            win = xp[:, ky:ky + H, kx:kx + W, :]
            dw[:, :, ky, kx] = np.einsum("nijo,nijc->oc", dy, win)
            dxp[:, ky:ky + H, kx:kx + W, :] += dy @ np.asarray(w[:, :, ky, kx], dtype=np.float64)
    return dxp[:, 1:H + 1, 1:W + 1], dw, dy.sum(axis=(0, 1, 2))


# ------------------------------------------------------------------ network
def layer_shapes():
    """(Cout, Cin) of the eight layers."""
    return [(HIDDEN, 1)] + [(HIDDEN, HIDDEN)] * 6 + [(1, HIDDEN)]


def flat_offsets():
    """Offsets of (w_l, c_l) in the flat parameter vector: for each layer its
    weights in (Cout, Cin, 3, 3) order, then its Cout biases."""
    off, o = [], 0
    for co, ci in layer_shapes():
        off.append((o, o + co * ci * 9))
        o += co * ci * 9 + co
    return off, o


def unflatten(theta):
    offs, total = flat_offsets()
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == total
    out = []
    for (ow, oc), (co, ci) in zip(offs, layer_shapes()):
        out.append((theta[ow:oc].reshape(co, ci, 3, 3), theta[oc:oc + co]))
    return out


def flatten(params):
    return np.concatenate([np.concatenate([w.ravel(), c.ravel()]) for w, c in params])


def forward(theta, b, bf16=False):
    """(u_hat, activations a_1 .. a_7) for the observation b (n, H, W)."""
    params = unflatten(theta)
    a = np.asarray(b, dtype=np.float64)[..., None]
    acts = []
    for l, (w, c) in enumerate(params):
        if bf16 and 0 < l < LAYERS - 1:
            w = round_bf16(w)
        z = conv3x3(a, w, c)
        if l == LAYERS - 1:
            return np.asarray(b, dtype=np.float64) + z[..., 0], acts
        a = np.maximum(z, 0.0)
        if bf16:
            a = round_bf16(a)
        acts.append(a)


def loss(u_hat, u_ref):
    d = np.asarray(u_hat, dtype=np.float64) - np.asarray(u_ref, dtype=np.float64)
    return 0.5 * float(np.sum(d * d)) / d.size


def backward(theta, b, u_ref, bf16=False):
    """(loss, d loss / d theta) by reverse mode through `forward`; with bf16
    the gradients with respect to the hidden activations are rounded to
    bfloat16 as the GPU path stores them."""
    params = unflatten(theta)
    u_hat, acts = forward(theta, b, bf16)
    n = u_hat.size
    l = loss(u_hat, u_ref)
    g = ((u_hat - np.asarray(u_ref, dtype=np.float64)) / n)[..., None]
    inputs = [np.asarray(b, dtype=np.float64)[..., None]] + acts
    grads = [None] * LAYERS
    for layer in range(LAYERS - 1, -1, -1):
        w, _ = params[layer]
        if bf16 and 0 < layer < LAYERS - 1:
            w = round_bf16(w)
        dx, dw, dc = conv3x3_backward(inputs[layer], w, g)
        grads[layer] = (dw, dc)
        if layer == 0:
            break
        g = dx * (inputs[layer] > 0)  # relu' of the layer below, from its output
        if bf16:
            g = round_bf16(g)
    return l, flatten(grads)


# -------------------------------------------------------------------- Adam
def adam_step(theta, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1) of step number `step` >= 1:
      m <- beta1 m + (1 - beta1) g;  v <- beta2 v + (1 - beta2) g^2
      theta <- theta - lr m_hat / (sqrt(v_hat) + eps),
      m_hat = m / (1 - beta1^step), v_hat = v / (1 - beta2^step)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
