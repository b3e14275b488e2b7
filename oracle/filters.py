"""Two-channel filter banks, derived in float64 from their defining polynomials.

Sec. I-B of the paper uses orthogonal wavelets (Haar, Daubechies) and Sec. I-C
the biorthogonal CDF 9/7 pair; it never prints taps.  Here the taps are derived
(never typed in):

* Daubechies with p vanishing moments: the halfband polynomial
  P_p(y) = sum_{k<p} C(p-1+k, k) y^k with y = sin^2(w/2) = (2 - z - 1/z)/4 is
  split by spectral factorisation; every root y_i gives a conjugate pair
  z_i, 1/z_i and the minimum-phase choice |z_i| < 1 goes to the scaling filter
  h(w) = (1 + w)^p * prod_i (1 - z_i w), w = z^-1, normalised to sum sqrt(2).
  "4-tap" is p = 2 (db2), "8-tap" is p = 4 (db4).
* CDF 9/7: the same P_4(y) is split between analysis and synthesis lowpass:
  both get cos^4(w/2); the real root of P_4 goes to the 7-tap synthesis
  lowpass, the complex pair to the 9-tap analysis lowpass.  Both are
  symmetric and normalised to sum sqrt(2).

Conventions (identical for every wavelet, so the orthogonal and biorthogonal
cases share one delay):
* all four filters live in arrays of one even length L, with L' = L - 1;
* orthogonal: dec_lo[k] = rec_lo[L-1-k];
* CDF 9/7: L = 10 (zero-padded), dec_lo occupies taps 1..9, rec_lo 1..7;
  with these placements the bank reconstructs with delay exactly L' (L = 9
  admits no placement with delay L' = 8 -- pinned by a test);
* highpass by modulation: rec_hi[k] = (-1)^k dec_lo[k],
  dec_hi[k] = (-1)^(k+1) rec_lo[k], which cancels aliasing for any lowpass pair
  and, for orthogonal filters, gives dec_hi[k] = rec_hi[L-1-k].
"""

from dataclasses import dataclass
from math import comb, sqrt

import numpy as np

WAVELETS = ("haar", "db2", "db4", "cdf97")


@dataclass(frozen=True)
class FilterBank:
    name: str
    L: int
    dec_lo: np.ndarray
    dec_hi: np.ndarray
    rec_lo: np.ndarray
    rec_hi: np.ndarray
    orthogonal: bool

    @property
    def Lp(self) -> int:
        return self.L - 1

    def dual_analysis(self):
        """Analysis filters of the dual frame: the synthesis filters reversed
        within the L-array (Eq. 3: W_zpd^* is analysis with the dual filters)."""
        return self.rec_lo[::-1].copy(), self.rec_hi[::-1].copy()


def daubechies_halfband(p: int) -> np.ndarray:
    """Coefficients (ascending powers of y) of P_p(y) = sum_k C(p-1+k,k) y^k."""
    return np.array([comb(p - 1 + k, k) for k in range(p)], dtype=np.float64)


def _y_to_zroot(y: complex) -> complex:
    # y = (2 - z - 1/z)/4  <=>  z^2 - (2 - 4y) z + 1 = 0; keep |z| < 1.
    b = 2.0 - 4.0 * y
    disc = np.sqrt(complex(b * b - 4.0))
    z1, z2 = (b + disc) / 2.0, (b - disc) / 2.0
    return z1 if abs(z1) < abs(z2) else z2


def daubechies_scaling(p: int) -> np.ndarray:
    """Minimum-phase Daubechies scaling filter with p vanishing moments."""
    P = daubechies_halfband(p)
    yroots = np.roots(P[::-1]) if p > 1 else np.array([])
    poly = np.array([1.0 + 0j])                  # ascending powers of w = z^-1
    for _ in range(p):
        poly = np.convolve(poly, [1.0, 1.0])
    for y in yroots:
        poly = np.convolve(poly, [1.0, -_y_to_zroot(complex(y))])
    h = poly.real
    assert np.allclose(poly.imag, 0.0, atol=1e-12)
    return h * (sqrt(2.0) / h.sum())


def _laurent_y():
    # y = sin^2(w/2) = (2 - z - 1/z)/4 as a symmetric 3-tap sequence
    return np.array([-0.25, 0.5, -0.25])


def cdf97_lowpass():
    """(analysis 9-tap, synthesis 7-tap) symmetric CDF 9/7 lowpass filters."""
    P = daubechies_halfband(4)                   # 1 + 4y + 10y^2 + 20y^3
    roots = np.roots(P[::-1])
    real_root = roots[np.argmin(np.abs(roots.imag))].real
    cplx = roots[np.argmax(roots.imag)]
    cos2 = np.array([0.25, 0.5, 0.25])           # cos^2(w/2) = (2 + z + 1/z)/4
    c4 = np.convolve(cos2, cos2)
    unit = np.array([0.0, 1.0, 0.0])
    syn7 = np.convolve(c4, unit - _laurent_y() / real_root)
    quad = np.convolve(unit - _laurent_y() / cplx, unit - _laurent_y() / np.conj(cplx))
    assert np.allclose(quad.imag, 0.0, atol=1e-12)
    ana9 = np.convolve(c4, quad.real)
    ana9 *= sqrt(2.0) / ana9.sum()
    syn7 = syn7 * (sqrt(2.0) / syn7.sum())
    return ana9, syn7


def _bank(name, L, dec_lo, rec_lo, orthogonal):
    k = np.arange(L)
    rec_hi = ((-1.0) ** k) * dec_lo
    dec_hi = ((-1.0) ** (k + 1)) * rec_lo
    return FilterBank(name, L, dec_lo, dec_hi, rec_lo, rec_hi, orthogonal)


def filter_bank(name: str) -> FilterBank:
    if name == "haar":
        rec_lo = np.array([1.0, 1.0]) / sqrt(2.0)
        return _bank(name, 2, rec_lo[::-1].copy(), rec_lo, True)
    if name in ("db2", "db4"):
        rec_lo = daubechies_scaling(int(name[2:]))
        return _bank(name, len(rec_lo), rec_lo[::-1].copy(), rec_lo, True)
    if name == "cdf97":
        ana9, syn7 = cdf97_lowpass()
        L = 10
        dec_lo = np.zeros(L)
        dec_lo[1:10] = ana9
        rec_lo = np.zeros(L)
        rec_lo[1:8] = syn7
        return _bank(name, L, dec_lo, rec_lo, False)
    raise ValueError(f"unknown wavelet {name!r}")
