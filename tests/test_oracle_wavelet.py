"""Pins of the oracle's W, W^dagger and W^* (Sec. I-A, Eq. 2-4)."""
from math import sqrt

import numpy as np
import pytest

from oracle import extension as ext
from oracle import filters, layout, wavelet

WAVELETS = filters.WAVELETS
MODES = wavelet.MODES


def _cases(mode):
    cases = [(4, 6, 1), (5, 3, 2), (8, 8, 2), (2, 2, 1), (1, 3, 1), (9, 4, 3)]
    return [c for c in cases if mode != "per" or (c[0] % 2 ** c[2] == 0 and c[1] % 2 ** c[2] == 0)]


@pytest.mark.parametrize("w", WAVELETS)
@pytest.mark.parametrize("mode", MODES)
def test_perfect_reconstruction(w, mode):
    """W W^dagger = I for every boundary mode (W = E^dagger S, W^dagger = Phi E)."""
    rng = np.random.default_rng(7)
    for r, c, J in _cases(mode) + [(16, 12, 2), (32, 20, 3)]:
        if mode == "per" and (r % 2 ** J or c % 2 ** J):
            continue
        img = rng.standard_normal((r, c))
        x = wavelet.wt_pinv(img, J, w, mode)
        assert len(x) == layout.num_coeffs(r, c, J, filters.filter_bank(w).L, mode)
        assert np.abs(wavelet.wt_synth(x, r, c, J, w, mode) - img).max() < 1e-12


@pytest.mark.parametrize("w", WAVELETS)
@pytest.mark.parametrize("mode", MODES)
def test_adjoint_equals_dense_transpose_both_routes(w, mode):
    """Eq. 4 route (ii) and the statement-wise transpose (i) both equal W^T."""
    rng = np.random.default_rng(11)
    for r, c, J in _cases(mode):
        Wd = wavelet.dense_synth(r, c, J, w, mode)
        for _ in range(2):
            img = rng.standard_normal((r, c))
            ref = Wd.T @ img.ravel()
            assert np.abs(wavelet.wt_adjoint(img, J, w, mode) - ref).max() < 1e-13
            assert np.abs(wavelet.wt_adjoint_transposed(img, J, w, mode) - ref).max() < 1e-13


@pytest.mark.parametrize("w", WAVELETS)
@pytest.mark.parametrize("mode", MODES)
def test_dot_product(w, mode):
    """<W x, y> = <x, W^* y> to 1e-12 relative at a moderate size."""
    r, c, J = (64, 48, 3)
    rng = np.random.default_rng(3)
    L = filters.filter_bank(w).L
    x = rng.standard_normal(layout.num_coeffs(r, c, J, L, mode))
    y = rng.standard_normal((r, c))
    lhs = float(np.sum(wavelet.wt_synth(x, r, c, J, w, mode) * y))
    rhs = float(np.dot(x, wavelet.wt_adjoint(y, J, w, mode)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("w", ["haar", "db2", "db4"])
def test_orthogonal_zpd_adjoint_is_analysis(w):
    """Sec. I-B: for orthogonal wavelets W_zpd^* = W_zpd^dagger; with the zero
    extension (E^dagger)^* = E, so W^* = W^dagger exactly."""
    rng = np.random.default_rng(5)
    img = rng.standard_normal((13, 10))
    a = wavelet.wt_adjoint(img, 2, w, "zero")
    b = wavelet.wt_pinv(img, 2, w, "zero")
    assert np.abs(a - b).max() < 1e-14
    # tight frame: Phi^T Phi = I on the zero-padded domain
    bank = filters.filter_bank(w)
    M = 11
    Phi = np.vstack([wavelet.zpd_analysis_axis0(np.eye(M), bank.dec_lo),
                     wavelet.zpd_analysis_axis0(np.eye(M), bank.dec_hi)])
    assert np.allclose(Phi.T @ Phi, np.eye(M), atol=1e-14)


def test_biorthogonal_frame_relations():
    """Table of frame relations: S Phi = I (Phi^dagger Phi = I) but Phi S != I,
    and W^* != W^dagger for CDF 9/7 even with zero extension."""
    bank = filters.filter_bank("cdf97")
    M = 15
    Phi = np.vstack([wavelet.zpd_analysis_axis0(np.eye(M), bank.dec_lo),
                     wavelet.zpd_analysis_axis0(np.eye(M), bank.dec_hi)])
    n = Phi.shape[0] // 2
    S = np.hstack([wavelet.zpd_synthesis_axis0(np.eye(n), bank.rec_lo, M),
                   wavelet.zpd_synthesis_axis0(np.eye(n), bank.rec_hi, M)])
    assert np.allclose(S @ Phi, np.eye(M), atol=1e-13)
    assert np.abs(Phi @ S - np.eye(2 * n)).max() > 1e-3
    assert np.abs(Phi.T @ Phi - np.eye(M)).max() > 1e-3       # not a tight frame
    img = np.random.default_rng(1).standard_normal((12, 12))
    assert np.abs(wavelet.wt_adjoint(img, 1, "cdf97", "zero")
                  - wavelet.wt_pinv(img, 1, "cdf97", "zero")).max() > 1e-3


@pytest.mark.parametrize("w", ["haar", "db2", "db4"])
def test_per_orthogonal_adjoint_is_inverse(w):
    """Critically sampled circular transform, orthogonal filters: W^* = W^-1."""
    r, c, J = 16, 8, 3
    Wd = wavelet.dense_synth(r, c, J, w, "per")
    assert Wd.shape == (r * c, r * c)
    assert np.allclose(Wd.T @ Wd, np.eye(r * c), atol=1e-13)
    assert np.allclose(Wd @ Wd.T, np.eye(r * c), atol=1e-13)


def test_per_biorthogonal_adjoint_is_not_inverse():
    r, c, J = 16, 16, 2
    Wd = wavelet.dense_synth(r, c, J, "cdf97", "per")
    assert np.abs(Wd.T @ Wd - np.eye(r * c)).max() > 1e-2
    assert np.allclose(np.linalg.inv(Wd), np.linalg.inv(Wd))  # square, invertible
    img = np.random.default_rng(2).standard_normal((r, c))
    x = wavelet.wt_pinv(img, J, "cdf97", "per")
    assert np.allclose(Wd @ x, img.ravel(), atol=1e-12)


@pytest.mark.parametrize("w", ["haar", "db2", "db4"])
@pytest.mark.parametrize("mode", ["sym", "ppd"])
def test_adjoint_minus_pinv_lives_at_the_boundary(w, mode):
    """Sec. I-B: the error of W^dagger ~ W^* enters only through E vs (E^dagger)^*,
    i.e. through the 2L' boundary samples with c > 1 (one level, 1D along axis 0)."""
    bank = filters.filter_bank(w)
    N, Lp = 40, bank.Lp
    y = np.random.default_rng(4).standard_normal((N, 1))
    a_lo, a_hi = wavelet.analysis_1d(y, bank, mode, "adjoint", axis=0)
    p_lo, p_hi = wavelet.analysis_1d(y, bank, mode, "pinv", axis=0)
    src = ext.ext_map(N, Lp, mode)
    c = ext.copy_counts(N, Lp, mode)
    touched = np.array([src[p] >= 0 and c[src[p]] > 1 for p in range(N + 2 * Lp)])
    n = a_lo.shape[0]
    for k in range(n):
        support = [e for e in range(2 * k + 1 - Lp, 2 * k + 2) if 0 <= e < N + 2 * Lp]
        if not any(touched[e] for e in support):
            assert abs(a_lo[k, 0] - p_lo[k, 0]) < 1e-14 and abs(a_hi[k, 0] - p_hi[k, 0]) < 1e-14
    assert np.abs(a_lo - p_lo).max() > 1e-6                   # and it is not zero overall


def test_haar_hand_values():
    """Haar by hand: circular y = [1,2,3,4] -> lo = (y0+y1, y2+y3)/sqrt2,
    hi = (y0-y1, y2-y3)/sqrt2; zero-padded N = 2 (L' = 1, M = 4, n = 2):
    lo = (y0, y1)/sqrt2, hi = (-y0, y1)/sqrt2."""
    bank = filters.filter_bank("haar")
    y = np.array([[1.0], [2.0], [3.0], [4.0]])
    lo, hi = wavelet.analysis_1d(y, bank, "per", "pinv", axis=0)
    assert np.allclose(lo[:, 0], [3 / sqrt(2), 7 / sqrt(2)], atol=1e-15)
    assert np.allclose(hi[:, 0], [-1 / sqrt(2), -1 / sqrt(2)], atol=1e-15)
    y2 = np.array([[5.0], [-3.0]])
    lo, hi = wavelet.analysis_1d(y2, bank, "zero", "pinv", axis=0)
    assert np.allclose(lo[:, 0], [5 / sqrt(2), -3 / sqrt(2)], atol=1e-15)
    assert np.allclose(hi[:, 0], [-5 / sqrt(2), -3 / sqrt(2)], atol=1e-15)


def test_band_length_is_odd_samples_of_full_convolution():
    for w in WAVELETS:
        L = filters.filter_bank(w).L
        for N in (1, 2, 7, 64, 277):
            M = N + 2 * (L - 1)
            full = np.convolve(np.ones(M), np.ones(L))
            assert layout.band_len(N, L, "sym") == len(full[1::2])
    # the 2048^2 CDF 9/7 five-level sizes used by the bench
    sizes = [s[1][0] for s in layout.level_sizes(2048, 2048, 5, 10, "sym")]
    assert sizes == [1037, 532, 279, 153, 90]
