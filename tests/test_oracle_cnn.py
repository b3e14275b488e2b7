"""Pins of the learned-warm-start oracle (oracle/cnn.py) against routes that
share none of its code: scipy's 2D correlation, the adjoint identity, exact
finite differences of a linear map, torch's bfloat16 cast, closed forms of
Adam's first step, and central differences of the whole network's loss."""
import numpy as np
import pytest
import scipy.signal
import torch

from oracle import cnn
from synthetic_inputs import he_normal_params, random_vector


def test_conv3x3_matches_scipy_correlate2d():
    """Each output channel is c[o] + sum_ci correlate2d(x[..., ci], w[o, ci],
    'same', zero fill): catches a flipped kernel, a transposed channel pair or
    an off-by-one halo."""
    x = random_vector((2, 7, 9, 3), 1)
    w = random_vector((4, 3, 3, 3), 2)
    c = random_vector(4, 3)
    y = cnn.conv3x3(x, w, c)
    for n in range(2):
        for o in range(4):
            ref = c[o] + sum(scipy.signal.correlate2d(x[n, :, :, ci], w[o, ci], mode="same", boundary="fill")
                             for ci in range(3))
            assert np.allclose(y[n, :, :, o], ref, rtol=1e-13, atol=1e-13)


def test_conv3x3_backward_adjoint_and_exact_differences():
    x = random_vector((2, 6, 5, 3), 4)
    w = random_vector((4, 3, 3, 3), 5)
    dy = random_vector((2, 6, 5, 4), 6)
    dx, dw, dc = cnn.conv3x3_backward(x, w, dy)
    # <conv(x), dy> = <x, dx>: dx is the adjoint applied to dy (no bias)
    assert np.isclose(np.sum(cnn.conv3x3(x, w) * dy), np.sum(x * dx), rtol=1e-13)
    # the map is linear in w and in c: one-sided differences are exact up to rounding
    e = np.zeros_like(w)
    for idx in [(0, 0, 0, 0), (3, 2, 2, 1), (1, 1, 1, 2)]:
        e[:] = 0.0
        e[idx] = 1.0
        d = np.sum((cnn.conv3x3(x, w + e) - cnn.conv3x3(x, w)) * dy)
        assert np.isclose(d, dw[idx], rtol=1e-11)
    assert np.allclose(dc, dy.sum(axis=(0, 1, 2)))
    c = np.zeros(4)
    c[2] = 1.0
    assert np.isclose(np.sum((cnn.conv3x3(x, w, c) - cnn.conv3x3(x, w)) * dy), dc[2], rtol=1e-12)


def test_round_bf16_ties_and_torch_cast():
    one = 1.0
    assert cnn.round_bf16(one) == 1.0
    assert cnn.round_bf16(1.0 + 2.0 ** -8) == 1.0                        # tie -> even (down)
    assert cnn.round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6         # tie -> even (up)
    assert cnn.round_bf16(1.0 + 2.0 ** -8 + 2.0 ** -12) == 1.0 + 2.0 ** -7
    assert cnn.round_bf16(-2.5) == -2.5
    v = random_vector(10000, 7) * np.exp(random_vector(10000, 8) * 5)
    ref = torch.tensor(v.astype(np.float32)).to(torch.bfloat16).double().numpy()
    assert np.array_equal(cnn.round_bf16(v), ref)


def test_flat_layout():
    offs, total = cnn.flat_offsets()
    assert total == 32 * 9 + 32 + 6 * (32 * 32 * 9 + 32) + 32 * 9 + 1
    assert offs[0] == (0, 288) and offs[1] == (320, 320 + 9216)
    theta = he_normal_params(cnn.layer_shapes(), 3)
    assert theta.size == total
    assert np.array_equal(cnn.flatten(cnn.unflatten(theta)), theta)


def test_network_gradient_central_differences():
    """d loss / d theta of the whole network against central differences in
    random unit directions (float64, no storage rounding)."""
    rows, cols = 9, 11
    b = random_vector((2, rows, cols), 11) * 0.3 + 0.5
    u = random_vector((2, rows, cols), 12) * 0.3 + 0.5
    theta = he_normal_params(cnn.layer_shapes(), 13, last_scale=1.0)
    l, g = cnn.backward(theta, b, u)
    assert np.isclose(l, cnn.loss(cnn.forward(theta, b)[0], u), rtol=1e-14)
    for s in range(3):
        d = random_vector(theta.size, 20 + s)
        d /= np.linalg.norm(d)   # a short step: no ReLU kink is crossed
        h = 1e-7
        fd = (cnn.loss(cnn.forward(theta + h * d, b)[0], u) - cnn.loss(cnn.forward(theta - h * d, b)[0], u)) / (2 * h)
        assert np.isclose(fd, g @ d, rtol=1e-5, atol=1e-10)


def test_bf16_storage_is_exact_on_representable_values():
    """With integer inputs, one +-1 weight per output channel and 128 pixels
    (so that d loss / d u_hat = integer / 128), every stored activation and
    gradient is a small dyadic number exact in bfloat16: the emulated storage
    rounding must then change nothing."""
    g = np.random.default_rng(5)
    params = []
    for co, ci in cnn.layer_shapes():
        w = np.zeros((co, ci, 3, 3))
        for o in range(co):
            w[o, g.integers(ci), g.integers(3), g.integers(3)] = g.choice([-1.0, 1.0])
        params.append((w, g.integers(-1, 2, size=co).astype(float)))
    theta = cnn.flatten(params)
    b = g.integers(0, 3, size=(2, 8, 8)).astype(float)
    u = g.integers(0, 3, size=(2, 8, 8)).astype(float)
    l0, g0 = cnn.backward(theta, b, u, bf16=False)
    l1, g1 = cnn.backward(theta, b, u, bf16=True)
    assert l0 == l1 and np.array_equal(g0, g1) and np.any(g0 != 0)


def test_relu_mask_uses_layer_output():
    """A unit whose pre-activation is negative passes no gradient: zeroing
    every weight and bias of layer 2 to a negative constant bias kills all
    gradients of layers 1 and 2's weights."""
    theta = he_normal_params(cnn.layer_shapes(), 14, last_scale=1.0)
    params = cnn.unflatten(theta)
    params[1] = (np.zeros_like(params[1][0]), -np.ones_like(params[1][1]))
    theta2 = cnn.flatten(params)
    b = random_vector((1, 6, 6), 15)
    _, g = cnn.backward(theta2, b, np.zeros((1, 6, 6)))
    offs, _ = cnn.flat_offsets()
    assert np.all(g[:offs[2][0]] == 0.0)


def test_adam_first_step_closed_form():
    """At step 1, m_hat = g and v_hat = g^2, so the update is lr g / (|g| + eps)."""
    theta = random_vector(50, 16)
    g = random_vector(50, 17)
    t1, m, v = cnn.adam_step(theta, g, np.zeros(50), np.zeros(50), 1, lr=0.01)
    assert np.allclose(theta - t1, 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    # a constant gradient keeps m_hat = g, v_hat = g^2 at every step
    t, m, v = theta, np.zeros(50), np.zeros(50)
    for k in range(1, 6):
        t_new, m, v = cnn.adam_step(t, g, m, v, k, lr=0.01)
        assert np.allclose(t - t_new, 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-9)
        t = t_new


def test_zero_last_layer_is_the_residual_identity():
    """With the last layer's weights zero, u_hat = b + c_8 exactly, whatever
    the hidden layers compute; d loss / d c_8 is then the mean of
    u_hat - u_ref, and every earlier parameter has zero gradient (the
    hidden activations do not reach the output)."""
    theta = he_normal_params(cnn.layer_shapes(), 31, last_scale=1.0)
    params = cnn.unflatten(theta)
    params[-1] = (np.zeros_like(params[-1][0]), np.array([0.25]))
    theta = cnn.flatten(params)
    b = random_vector((2, 7, 9), 32)
    u = random_vector((2, 7, 9), 33)
    u_hat, _ = cnn.forward(theta, b)
    assert np.array_equal(u_hat, b + 0.25)
    _, g = cnn.backward(theta, b, u)
    offs, _ = cnn.flat_offsets()
    assert np.isclose(g[-1], np.mean(u_hat - u), rtol=1e-13)
    assert np.all(g[:offs[-1][0]] == 0.0)


def test_first_layer_gradient_matches_its_own_definition():
    """Layer 1's weight gradient is sum_p dz_1[p][o] b[p + offset]: rebuilt
    here from the forward's activations and an independent backward through
    the last layers with scipy's correlation, on a tiny network whose
    middle layers are identities (one centre tap per channel)."""
    rng = np.random.default_rng(34)
    params = []
    for i, (co, ci) in enumerate(cnn.layer_shapes()):
        w = np.zeros((co, ci, 3, 3))
        if 0 < i < cnn.LAYERS - 1:
            for o in range(co):
                w[o, o, 1, 1] = 1.0        # identity on each channel
        else:
            w[...] = rng.standard_normal(w.shape) * 0.3
        params.append((w, np.zeros(co)))
    theta = cnn.flatten(params)
    b = np.abs(random_vector((1, 6, 8), 35)) + 0.1
    u = random_vector((1, 6, 8), 36)
    u_hat, acts = cnn.forward(theta, b)
    _, g = cnn.backward(theta, b, u)
    # middle layers pass a_1 through unchanged where it is positive, so
    # d l / d a_1 = [a_1 > 0] conv_8^T(d l / d u_hat); then dz_1 = that masked again
    dout = (u_hat - u)[0] / u_hat.size
    w8 = params[-1][0][0]                              # (32, 3, 3)
    a1 = acts[0][0]
    dz1 = np.stack([scipy.signal.convolve2d(dout, w8[c], mode="same") for c in range(32)], axis=-1) * (a1 > 0)
    bp = np.pad(b[0], 1)
    want = np.zeros((32, 3, 3))
    for dy in range(3):
        for dx in range(3):
            want[:, dy, dx] = np.einsum("ijo,ij->o", dz1, bp[dy:dy + 6, dx:dx + 8])
    offs, _ = cnn.flat_offsets()
    assert np.allclose(g[offs[0][0]:offs[0][1]].reshape(32, 3, 3), want, rtol=1e-10, atol=1e-14)
