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
