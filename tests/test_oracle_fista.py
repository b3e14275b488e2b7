"""Pins of the oracle's FISTA, gradient and step size (Eq. 1, Sec. I-B)."""
import numpy as np
import pytest

from oracle import blur, filters, fista, layout, wavelet
from synthetic_inputs import gaussian_noise, piecewise_smooth_image, random_taps, random_vector


def _problem(rows=16, cols=12, levels=2, w="db2", mode="sym", k=5, lam=1e-3, seed=0, psf=None):
    p = blur.gaussian_psf(k, 1.0) if psf is None else psf
    img = piecewise_smooth_image(rows, cols, seed)
    b = blur.blur(img, p, p, mode if mode != "ppd" else "per") + gaussian_noise((rows, cols), seed + 1)
    return fista.Problem(rows, cols, levels, w, mode, p, p, mode if mode in blur.BCS else "per", b, lam)


def test_identity_blur_orthogonal_per_closed_form():
    """R = I and W orthogonal (circular): F(x) = 1/2||x - W^T b||^2 + lam||x||_1,
    whose minimiser is soft(W^T b, lam); with L_f = 1 FISTA lands on it in one
    iteration and stays."""
    prob = _problem(rows=16, cols=16, levels=3, w="db2", mode="per", psf=np.array([1.0]), lam=0.05)
    xstar = fista.soft(wavelet.wt_adjoint(prob.b, 3, "db2", "per"), 0.05)
    x1, _ = fista.fista(prob, 1.0, 1)
    assert np.abs(x1 - xstar).max() < 1e-14
    x5, _ = fista.fista(prob, 1.0, 5)
    assert np.abs(x5 - xstar).max() < 1e-14
    assert 0.1 < np.mean(xstar == 0) < 0.99                   # the threshold is active


def test_gradient_finite_difference():
    prob = _problem(mode="sym", w="cdf97", levels=1, rows=10, cols=9)
    C = layout.num_coeffs(10, 9, 1, 10, "sym")
    x = random_vector(C, 3)
    g, f0 = prob.grad(x)
    d = random_vector(C, 4)
    eps = 1e-6

    def f(z):
        res = prob.A(z) - prob.b
        return 0.5 * np.sum(res * res)
    fd = (f(x + eps * d) - f(x - eps * d)) / (2 * eps)
    assert abs(fd - np.dot(g, d)) < 1e-7 * max(1.0, abs(fd))
    assert abs(f0 - f(x)) < 1e-12 * f0


def test_power_iteration_matches_dense_spectrum():
    prob = _problem(rows=8, cols=6, levels=1, w="db2", mode="sym", k=3)
    C = layout.num_coeffs(8, 6, 1, 4, "sym")
    A = np.zeros((48, C))
    for i in range(C):
        e = np.zeros(C)
        e[i] = 1.0
        A[:, i] = prob.A(e).ravel()
    lam_max = np.linalg.eigvalsh(A.T @ A).max()
    est = fista.power_iteration(prob, random_vector(C, 9), iters=400)
    assert abs(est - lam_max) < 1e-8 * lam_max
    assert abs(fista.lipschitz(prob, random_vector(C, 9), iters=400) - 1.01 * lam_max) < 1e-7


def test_beck_teboulle_rate_bound():
    """F(x_k) - F* <= 2 L ||x_0 - x*||^2 / (k+1)^2 for every k."""
    prob = _problem(rows=16, cols=16, levels=2, w="db2", mode="sym", lam=2e-3)
    C = layout.num_coeffs(16, 16, 2, 4, "sym")
    L = fista.lipschitz(prob, random_vector(C, 1), iters=100)
    xstar, _ = fista.fista(prob, L, 3000)
    Fstar = prob.objective(xstar)
    _, hist = fista.fista(prob, L, 60, record_every=1)
    for k, Fk in hist:
        assert Fk - Fstar <= 2 * L * np.sum(xstar ** 2) / (k + 1) ** 2 + 1e-12


def test_objective_and_soft_threshold():
    v = np.array([-3.0, -1.0, -0.5, 0.0, 0.5, 1.0, 2.0])
    assert np.array_equal(fista.soft(v, 1.0), [-2.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0])
    prob = _problem()
    C = layout.num_coeffs(16, 12, 2, 4, "sym")
    x = random_vector(C, 2)
    res = blur.blur(wavelet.wt_synth(x, 16, 12, 2, "db2", "sym"), prob.p_rows, prob.p_cols, "sym") - prob.b
    assert abs(prob.objective(x) - (0.5 * np.sum(res ** 2) + 1e-3 * np.abs(x).sum())) < 1e-12
    assert abs(fista.t_next(1.0) - (1 + np.sqrt(5)) / 2) < 1e-15
