"""Pins of the oracle's convolution gradients (Sec. II, Eq. 5)."""
import os

import numpy as np
import pytest

from oracle import conv

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "conv_k3_n5.txt")


def _golden():
    mats = {"H": [], "S": [], "G": []}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        tag, *cells = line.split()
        mats[tag].append([-1 if c == "." else int(c) for c in cells])
    return {k: np.array(v) for k, v in mats.items()}


def _fill(pattern, vals):
    out = np.zeros(pattern.shape)
    ok = pattern >= 0
    out[ok] = np.asarray(vals)[pattern[ok]]
    return out


def test_paper_k3_n5_matrices_exact():
    g = _golden()
    h = np.array([2.0, -1.0, 3.0])
    s = np.array([1.0, 4.0, -2.0, 5.0, 3.0])
    r = np.array([1.0, -2.0, 0.0, 7.0, 2.0, -1.0, 4.0])
    H = _fill(g["H"], h)
    S = _fill(g["S"], s)
    G = _fill(g["G"], s)
    x = conv.conv_full(h, s)
    assert np.array_equal(x, H @ s) and np.array_equal(x, S @ h)
    assert np.array_equal(conv.conv_matrix_S(s, 3), S) and np.array_equal(conv.conv_matrix_H(h, 5), H)
    gh, gs = conv.conv_adjoint(s, h, r)
    assert np.array_equal(gh, G @ r)                 # grad_h = S^T r
    assert np.array_equal(G, S.T)
    assert np.array_equal(gs, H.T @ r)               # grad_s = H^T r


def test_matches_numpy_correlate_and_matlab_form():
    rng = np.random.default_rng(0)
    N, K = 37, 6
    s, h = rng.standard_normal(N), rng.standard_normal(K)
    r = rng.standard_normal(N + K - 1)
    gh, gs = conv.conv_adjoint(s, h, r)
    # conv(r, conj(s(end:-1:1)), 'valid') of Sec. II
    assert np.allclose(gh, np.convolve(r, s[::-1], mode="valid"), atol=1e-13)
    assert np.allclose(gs, np.convolve(r, h[::-1], mode="valid"), atol=1e-13)
    assert np.allclose(conv.conv_full(h, s), np.convolve(h, s), atol=1e-14)


@pytest.mark.parametrize("N,K", [(1, 1), (1, 4), (5, 1), (3, 9), (64, 8)])
def test_dense_transpose_and_batch(N, K):
    rng = np.random.default_rng(N * 100 + K)
    s, h = rng.standard_normal((3, N)), rng.standard_normal((3, K))
    r = rng.standard_normal((3, N + K - 1))
    gh, gs = conv.conv_adjoint(s, h, r)
    for b in range(3):
        assert np.allclose(gh[b], conv.conv_matrix_S(s[b], K).T @ r[b], atol=1e-13)
        assert np.allclose(gs[b], conv.conv_matrix_H(h[b], N).T @ r[b], atol=1e-13)


def test_finite_difference_gradient():
    rng = np.random.default_rng(5)
    N, K = 20, 5
    s, h, x = rng.standard_normal(N), rng.standard_normal(K), rng.standard_normal(N + K - 1)

    def f(hh, ss):
        res = conv.conv_full(hh, ss) - x
        return 0.5 * np.sum(res * res)
    r = conv.conv_full(h, s) - x
    gh, gs = conv.conv_adjoint(s, h, r)
    eps = 1e-6
    for n in range(K):
        e = np.zeros(K)
        e[n] = eps
        assert abs((f(h + e, s) - f(h - e, s)) / (2 * eps) - gh[n]) < 1e-7
    for m in range(0, N, 3):
        e = np.zeros(N)
        e[m] = eps
        assert abs((f(h, s + e) - f(h, s - e)) / (2 * eps) - gs[m]) < 1e-7


def test_bce_gradient_finite_differences_and_parts():
    """Eq. 6: the gradient of the smooth multichannel objective matches central
    differences; D^T is the transpose of the dense difference matrix; the
    Huber function is quadratic inside [-delta, delta] and linear outside."""
    rng = np.random.default_rng(11)
    C, N, K, lam_tv, delta = 2, 9, 5, 0.3, 0.1
    s, H = rng.standard_normal(N), rng.standard_normal((C, K))
    X = rng.standard_normal((C, N + K - 1))
    gh, gs = conv.bce_gradient(s, H, X, lam_tv, delta)
    eps = 1e-6
    for c in range(C):
        for j in range(K):
            Hp, Hm = H.copy(), H.copy()
            Hp[c, j] += eps
            Hm[c, j] -= eps
            fd = (conv.bce_smooth(s, Hp, X, lam_tv, delta) - conv.bce_smooth(s, Hm, X, lam_tv, delta)) / (2 * eps)
            assert abs(fd - gh[c, j]) <= 1e-6 * (1 + abs(fd))
    for m in range(N):
        sp, sm = s.copy(), s.copy()
        sp[m] += eps
        sm[m] -= eps
        fd = (conv.bce_smooth(sp, H, X, lam_tv, delta) - conv.bce_smooth(sm, H, X, lam_tv, delta)) / (2 * eps)
        assert abs(fd - gs[m]) <= 1e-6 * (1 + abs(fd))
    D = np.diff(np.eye(K), axis=0)  # (D h)[j] = h[j+1] - h[j]
    v = rng.standard_normal(K - 1)
    assert np.allclose(conv.tv_diff(H[0]), D @ H[0]) and np.allclose(conv.tv_diff_adjoint(v), D.T @ v)
    z = np.array([-0.3, -0.1, 0.05, 0.1, 0.2])
    assert np.allclose(conv.huber(z, 0.1), [0.1 * (0.3 - 0.05), 0.005, 0.00125, 0.005, 0.1 * (0.2 - 0.05)])
