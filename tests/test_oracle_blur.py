"""Pins of the oracle's R and R^* against library routines and closed forms."""
import numpy as np
import pytest
from scipy.signal import convolve2d

from oracle import blur
from synthetic_inputs import random_taps

BCS = blur.BCS
PAD = {"zero": "constant", "sym": "symmetric", "per": "wrap"}


def test_gaussian_psf_closed_form():
    p = blur.gaussian_psf(9, 1.5)
    c = 4.0
    ref = np.exp(-((np.arange(9) - c) ** 2) / (2 * 1.5 ** 2))
    assert np.allclose(p, ref / ref.sum(), atol=1e-16)
    assert abs(p.sum() - 1.0) < 1e-15 and np.allclose(p, p[::-1])


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("shape,k", [((12, 9), 5), ((20, 17), 9), ((7, 11), 3),
                                     ((2, 3), 9), ((1, 4), 7), ((3, 1), 15), ((5, 2), 11)])
def test_blur_is_valid_2d_convolution_of_padded_image(bc, shape, k):
    """R u = 'valid' 2D convolution (scipy) of the image padded by r with numpy's
    constant / half-point symmetric / wrap modes, for a non-separable loop over the
    full 2D PSF outer(p_r, p_c).  The last four shapes are smaller than the radius,
    where numpy's padding repeats the reflection (or the wrap) and so pins the
    repeated branch of the extension (Sec. I-A, reading C1)."""
    rng = np.random.default_rng(0)
    u = rng.standard_normal(shape)
    pr, pc = random_taps(k, 1), random_taps(k, 2)
    r = k // 2
    up = np.pad(u, r, mode=PAD[bc])
    ref = convolve2d(up, np.outer(pr, pc), mode="valid")
    assert np.abs(blur.blur(u, pr, pc, bc) - ref).max() < 1e-13


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("shape,kr,kc", [((6, 5), 3, 5), ((9, 8), 7, 3), ((3, 4), 9, 7), ((1, 2), 5, 3)])
def test_adjoint_is_dense_transpose(bc, shape, kr, kc):
    """R^* equals the transpose of the dense R, for asymmetric PSFs (so R^* != R),
    including images smaller than the PSF (repeated reflection / wrap)."""
    pr, pc = random_taps(kr, 3), random_taps(kc, 4)
    Rm = blur.dense_blur(*shape, pr, pc, bc)
    rng = np.random.default_rng(1)
    for _ in range(2):
        v = rng.standard_normal(shape)
        assert np.abs(blur.blur_adjoint(v, pr, pc, bc).ravel() - Rm.T @ v.ravel()).max() < 1e-14
    if min(shape) >= 3:
        assert np.abs(Rm - Rm.T).max() > 1e-3


@pytest.mark.parametrize("bc", BCS)
def test_symmetric_psf_self_adjoint(bc):
    p = blur.gaussian_psf(7, 1.2)
    Rm = blur.dense_blur(10, 9, p, p, bc)
    assert np.abs(Rm - Rm.T).max() < 1e-15


@pytest.mark.parametrize("bc", ["sym", "per"])
def test_normalised_psf_preserves_constants(bc):
    p = random_taps(9, 5)
    out = blur.blur(np.ones((11, 13)), p, p[::-1].copy(), bc)
    assert np.abs(out - 1.0).max() < 1e-14


def test_per_is_circular_convolution_fft():
    rng = np.random.default_rng(2)
    u = rng.standard_normal((16, 12))
    pr, pc = random_taps(5, 6), random_taps(3, 7)
    ker = np.zeros((16, 12))
    for a in range(5):
        for b in range(3):
            ker[(a - 2) % 16, (b - 1) % 12] = pr[a] * pc[b]
    ref = np.real(np.fft.ifft2(np.fft.fft2(u) * np.fft.fft2(ker)))
    assert np.abs(blur.blur(u, pr, pc, "per") - ref).max() < 1e-13


def test_blur_normal_gradient_finite_difference():
    rng = np.random.default_rng(3)
    u = rng.standard_normal((8, 7))
    b = rng.standard_normal((8, 7))
    pr, pc = random_taps(5, 8), random_taps(3, 9)
    g, f0 = blur.blur_normal(u, b, pr, pc, "sym")
    d = rng.standard_normal((8, 7))
    eps = 1e-6
    fp = blur.blur_normal(u + eps * d, b, pr, pc, "sym")[1]
    fm = blur.blur_normal(u - eps * d, b, pr, pc, "sym")[1]
    assert abs((fp - fm) / (2 * eps) - np.sum(g * d)) < 1e-7 * max(1.0, abs(np.sum(g * d)))
