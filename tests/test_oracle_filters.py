"""Pins of the oracle's filter banks against their defining properties."""
from math import comb, sqrt

import numpy as np
import pytest

from oracle import filters, wavelet


def test_haar_closed_form():
    b = filters.filter_bank("haar")
    assert np.allclose(b.rec_lo, [1 / sqrt(2), 1 / sqrt(2)], atol=0, rtol=1e-15)
    assert np.allclose(b.dec_hi, [-1 / sqrt(2), 1 / sqrt(2)], atol=1e-16)


def test_db2_textbook_closed_form():
    # Daubechies' 4-tap scaling filter in closed form: (1+-sqrt3), (3+-sqrt3) over 4 sqrt2
    s3 = sqrt(3.0)
    ref = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4 * sqrt(2.0))
    assert np.allclose(filters.filter_bank("db2").rec_lo, ref, atol=1e-15)


@pytest.mark.parametrize("name,p", [("haar", 1), ("db2", 2), ("db4", 4)])
def test_orthonormal_and_vanishing_moments(name, p):
    b = filters.filter_bank(name)
    h = b.rec_lo
    assert len(h) == 2 * p
    for m in range(-(p - 1), p):              # sum_k h[k] h[k+2m] = delta_m
        s = sum(h[k] * h[k + 2 * m] for k in range(len(h)) if 0 <= k + 2 * m < len(h))
        assert abs(s - (1.0 if m == 0 else 0.0)) < 1e-14
    k = np.arange(len(h))
    for q in range(p):                        # highpass annihilates polynomials of degree < p
        assert abs(np.sum(b.rec_hi * k ** q)) < 1e-11 * max(1, (len(h)) ** q)
        assert abs(np.sum(b.dec_hi * k ** q)) < 1e-11 * max(1, (len(h)) ** q)
    assert np.allclose(b.dec_lo, h[::-1]) and np.allclose(b.dec_hi, b.rec_hi[::-1])


def test_db4_minimum_phase():
    h = filters.filter_bank("db4").rec_lo
    zeros = np.roots(h)                       # zeros of H in z (polynomial in z^-1 read as z)
    not_at_minus1 = zeros[np.abs(zeros + 1) > 1e-3]
    assert len(not_at_minus1) == 3
    assert np.all(np.abs(not_at_minus1) < 1.0)


def test_daubechies_halfband_polynomial():
    # P_p(y) of degree p-1 with binomial coefficients; p = 4 gives 1 + 4y + 10y^2 + 20y^3
    assert list(filters.daubechies_halfband(4)) == [1, 4, 10, 20]
    assert list(filters.daubechies_halfband(2)) == [comb(1, 0), comb(2, 1)]


def test_cdf97_structure():
    b = filters.filter_bank("cdf97")
    assert b.L == 10 and not b.orthogonal
    ana, syn = b.dec_lo[1:10], b.rec_lo[1:8]
    assert b.dec_lo[0] == 0 and np.all(b.rec_lo[8:] == 0) and b.rec_lo[0] == 0
    assert np.allclose(ana, ana[::-1], atol=1e-15) and np.allclose(syn, syn[::-1], atol=1e-15)
    assert abs(ana.sum() - sqrt(2)) < 1e-14 and abs(syn.sum() - sqrt(2)) < 1e-14
    k = np.arange(10)
    for q in range(4):                        # 4 vanishing moments on both sides
        assert abs(np.sum(b.dec_hi * k ** q)) < 1e-10 * 10 ** q
        assert abs(np.sum(b.rec_hi * k ** q)) < 1e-10 * 10 ** q
    # dec_lo has exactly the 9 taps, rec_lo the 7 taps
    assert np.count_nonzero(np.abs(b.dec_lo) > 1e-12) == 9
    assert np.count_nonzero(np.abs(b.rec_lo) > 1e-12) == 7


@pytest.mark.parametrize("name", filters.WAVELETS)
def test_product_filter_halfband_with_delay_Lprime(name):
    """Perfect reconstruction in the filter domain: the odd samples of
    rec_lo * dec_lo vanish except the one at the delay L' (where it is 1)."""
    b = filters.filter_bank(name)
    P = np.convolve(b.rec_lo, b.dec_lo)
    for n in range(1, len(P), 2):
        assert abs(P[n] - (1.0 if n == b.Lp else 0.0)) < 1e-14


def _zpd_pr_error(dec_lo, rec_lo, M=23):
    L = len(dec_lo)
    k = np.arange(L)
    rec_hi = ((-1.0) ** k) * dec_lo
    dec_hi = ((-1.0) ** (k + 1)) * rec_lo
    err = 0.0
    for t in range(M):
        z = np.zeros((M, 1))
        z[t] = 1.0
        lo = wavelet.zpd_analysis_axis0(z, dec_lo)
        hi = wavelet.zpd_analysis_axis0(z, dec_hi)
        zr = wavelet.zpd_synthesis_axis0(lo, rec_lo, M) + wavelet.zpd_synthesis_axis0(hi, rec_hi, M)
        err = max(err, float(np.abs(zr - z).max()))
    return err


def test_cdf97_needs_length_10():
    """Reading of 'L = maximum length of the analysis filters' for CDF 9/7: in a
    9-array no placement of the 9- and 7-tap filters reconstructs with the
    delay L' = 8 that the extension by L' implies; in the 10-array the chosen
    placement does (delay 9)."""
    ana, syn = filters.cdf97_lowpass()
    for o7 in range(3):
        d = np.zeros(9)
        d[:] = ana
        r = np.zeros(9)
        r[o7:o7 + 7] = syn
        assert _zpd_pr_error(d, r) > 1e-3
    b = filters.filter_bank("cdf97")
    assert _zpd_pr_error(b.dec_lo, b.rec_lo) < 1e-13
