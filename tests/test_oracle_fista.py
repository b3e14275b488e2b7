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


def test_pinv_in_place_of_adjoint_fails_to_minimise():
    """The paper's comparison (Sec. I-B, I-C): FISTA with W^dagger standing in
    for W^* no longer descends F for a biorthogonal transform with symmetric
    boundaries, while for an orthogonal transform with circular (or zero)
    boundaries W^dagger = W^* and the two runs coincide."""
    from oracle import blur as ob
    from oracle import fista as ofista
    from oracle.layout import num_coeffs
    from synthetic_inputs import gaussian_noise, piecewise_smooth_image, random_vector
    r, c, lam = 48, 40, 2e-3
    p = ob.gaussian_psf(7, 1.2)
    out = {}
    for w, mode, bc, L_len in [("cdf97", "sym", "sym", 10), ("db2", "per", "per", 4)]:
        b = ob.blur(piecewise_smooth_image(r, c, 5), p, p, bc) + gaussian_noise((r, c), 6)
        exact = ofista.Problem(r, c, 2, w, mode, p, p, bc, b, lam)
        pinv = ofista.Problem(r, c, 2, w, mode, p, p, bc, b, lam, gradient="pinv")
        L = ofista.lipschitz(exact, random_vector(num_coeffs(r, c, 2, L_len, mode), 1), 30)
        assert ofista.lipschitz(pinv, random_vector(num_coeffs(r, c, 2, L_len, mode), 1), 30) == L
        _, he = ofista.fista(exact, L, 150, record_every=150)
        _, hp = ofista.fista(pinv, L, 150, record_every=150)
        out[w] = (he[-1][1], hp[-1][1])
    fe, fp = out["cdf97"]
    assert fp > 1.1 * fe  # 1.42 vs 1.18 at this size
    fe, fp = out["db2"]
    assert abs(fp - fe) <= 1e-12 * fe
