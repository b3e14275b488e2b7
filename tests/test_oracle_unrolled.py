"""Pins of the oracle's derivative machinery (float64, central differences):
the Gaussian taps' derivative in sigma, dR/dsigma, and the reverse mode of
unrolled FISTA with respect to lambda, sigma and b (differentiation of the
solve of Eq. 1 through the chain rule of Sec. I)."""
import ctypes as C

import numpy as np
import pytest

from oracle import blur as oblur
from oracle import fista as ofista
from oracle import unrolled as ounr
from oracle.filters import filter_bank
from oracle.layout import num_coeffs
from synthetic_inputs import gaussian_noise, piecewise_smooth_image, random_vector


@pytest.mark.parametrize("k,sigma", [(5, 1.0), (9, 1.7), (15, 3.0), (1, 0.5)])
def test_gaussian_dsigma_central_differences(k, sigma):
    h = 1e-5 * sigma
    fd = (oblur.gaussian_psf(k, sigma + h) - oblur.gaussian_psf(k, sigma - h)) / (2 * h)
    an = oblur.gaussian_psf_dsigma(k, sigma)
    assert np.allclose(an, fd, rtol=1e-7, atol=1e-12)
    assert abs(an.sum()) < 1e-14  # the taps stay normalised


@pytest.mark.parametrize("bc", ["zero", "sym", "per"])
def test_dR_dsigma_central_differences(bc):
    k, sigma, h = 7, 1.3, 1e-5
    u = random_vector((11, 14), 3)
    S = ounr.Setup(11, 14, 1, "db2", "sym", k, sigma, bc, np.zeros((11, 14)), 0.0, 1.0)
    fd = (oblur.blur(u, *(2 * [oblur.gaussian_psf(k, sigma + h)]), bc)
          - oblur.blur(u, *(2 * [oblur.gaussian_psf(k, sigma - h)]), bc)) / (2 * h)
    assert np.allclose(S.dR(u), fd, rtol=1e-7, atol=1e-10)


def _setup(rows, cols, levels, wavelet, mode, bc, k, sigma, lam, seed, L=None):
    img = piecewise_smooth_image(rows, cols, seed)
    q = oblur.gaussian_psf(k, sigma)
    b = oblur.blur(img, q, q, bc) + gaussian_noise((rows, cols), seed + 1, 1e-2)
    nco = num_coeffs(rows, cols, levels, filter_bank(wavelet).L, mode)
    if L is None:
        prob = ofista.Problem(rows, cols, levels, wavelet, mode, q, q, bc, b, lam)
        L = ofista.lipschitz(prob, np.random.default_rng(seed).standard_normal(nco), iters=30)
    return ounr.Setup(rows, cols, levels, wavelet, mode, k, sigma, bc, b, lam, L), img, nco


@pytest.mark.parametrize("wavelet,mode,bc", [("db2", "sym", "sym"), ("cdf97", "sym", "sym"), ("db2", "per", "per")])
def test_unrolled_reverse_mode_central_differences(wavelet, mode, bc):
    rows = cols = 24
    S, img, nco = _setup(rows, cols, 2, wavelet, mode, bc, 5, 1.2, 0.02, 7)
    steps = 6
    loss, dlam, dsig, db = ounr.unrolled_grads(S, steps, img, nco)
    assert np.isclose(loss, ounr.unrolled_loss(S, steps, img, nco), rtol=1e-14)

    def at(lam=None, sigma=None, b=None):
        T = ounr.Setup(rows, cols, 2, wavelet, mode, 5, S.sigma if sigma is None else sigma, bc,
                       S.b if b is None else b, S.lam if lam is None else lam, S.L)
        return ounr.unrolled_loss(T, steps, img, nco)

    h = 1e-6
    fd_lam = (at(lam=S.lam + h) - at(lam=S.lam - h)) / (2 * h)
    fd_sig = (at(sigma=S.sigma + h) - at(sigma=S.sigma - h)) / (2 * h)
    d = random_vector((rows, cols), 11)
    fd_b = (at(b=S.b + h * d) - at(b=S.b - h * d)) / (2 * h)
    assert abs(dlam - fd_lam) <= 1e-6 * max(1.0, abs(fd_lam)), (dlam, fd_lam)
    assert abs(dsig - fd_sig) <= 1e-6 * max(1.0, abs(fd_sig)), (dsig, fd_sig)
    assert abs(float(np.sum(db * d)) - fd_b) <= 1e-6 * max(1.0, abs(fd_b)), (np.sum(db * d), fd_b)
    assert abs(dlam) > 1e-3 and abs(dsig) > 1e-3  # the pins are not vacuous


def test_library_gaussian_taps_match_the_oracle():
    """The library's host routine (no GPU needed) against the definition."""
    from paper_1707_02018_gb300 import _lib
    lib = _lib.load()
    for k, sigma in [(15, 3.0), (9, 1.7), (1, 0.4)]:
        taps, dt = (C.c_double * k)(), (C.c_double * k)()
        assert lib.adjwt_gaussian_taps(k, sigma, taps, dt) == 0
        assert np.allclose(list(taps), oblur.gaussian_psf(k, sigma), rtol=1e-14, atol=1e-17)
        assert np.allclose(list(dt), oblur.gaussian_psf_dsigma(k, sigma), rtol=1e-12, atol=1e-15)
    taps = (C.c_double * 4)()
    assert lib.adjwt_gaussian_taps(4, 1.0, taps, None) != 0
    assert lib.adjwt_gaussian_taps(5, 0.0, taps, None) != 0
