"""Full linear convolution and the two gradients of Sec. II (Eq. 5).

x_est = h * s (zero boundary, "full", length N + K - 1), with s of length N and
h of length K.  For f(h, s) = 1/2 ||h * s - x||^2 and residual r = h * s - x:

    grad_h f = S^T r:   grad_h[n] = sum_{k=0}^{N-1} s[k] r[k+n],  n = 0..K-1
    grad_s f = H^T r:   grad_s[m] = sum_{k=0}^{K-1} h[k] r[k+m],  m = 0..N-1

(the cross-correlations displayed after the two matrix forms of the
convolution; signals are real so the conjugation is a no-op).  The gradients
are returned unscaled (S^T r, no factor 2 for the unhalved Eq. 6 objective).
"""

import numpy as np


def conv_full(h, s):
    """x_est[m] = sum_k h[k] s[m-k], m = 0..N+K-2 (batched over leading axes)."""
    h = np.asarray(h, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    K, N = h.shape[-1], s.shape[-1]
    out = np.zeros(np.broadcast_shapes(h.shape[:-1], s.shape[:-1]) + (N + K - 1,))
    for k in range(K):
        out[..., k:k + N] += h[..., k:k + 1] * s
    return out


def conv_adjoint(s, h, r):
    """(grad_h, grad_s) for batched rows: s (..., N), h (..., K), r (..., N+K-1)."""
    s = np.asarray(s, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    N, K = s.shape[-1], h.shape[-1]
    assert r.shape[-1] == N + K - 1
    grad_h = np.zeros(h.shape)
    for n in range(K):
        grad_h[..., n] = np.sum(s * r[..., n:n + N], axis=-1)
    grad_s = np.zeros(s.shape)
    for k in range(K):
        grad_s += h[..., k:k + 1] * r[..., k:k + N]
    return grad_h, grad_s


def conv_matrix_S(s, K):
    """The paper's second matrix form: x_est = S h, S[m, k] = s[m-k]."""
    s = np.asarray(s, dtype=np.float64)
    N = len(s)
    S = np.zeros((N + K - 1, K))
    for k in range(K):
        S[k:k + N, k] = s
    return S


def conv_matrix_H(h, N):
    """The paper's first matrix form: x_est = H s, H[m, k] = h[m-k]."""
    h = np.asarray(h, dtype=np.float64)
    K = len(h)
    H = np.zeros((N + K - 1, N))
    for k in range(N):
        H[k:k + K, k] = h
    return H


def huber(z, delta):
    """L_delta(z) = z^2/2 for |z| <= delta, delta (|z| - delta/2) otherwise (Sec. II)."""
    z = np.asarray(z, dtype=np.float64)
    a = np.abs(z)
    return np.where(a <= delta, 0.5 * z * z, delta * (a - 0.5 * delta))


def huber_grad(z, delta):
    return np.clip(np.asarray(z, dtype=np.float64), -delta, delta)


def tv_diff(h):
    """D h: consecutive differences (D h)[j] = h[j+1] - h[j], j = 0..K-2."""
    h = np.asarray(h, dtype=np.float64)
    return h[..., 1:] - h[..., :-1]


def tv_diff_adjoint(v):
    """D^T v for v of length K-1: (D^T v)[j] = v[j-1] - v[j] with v[-1] = v[K-1] = 0."""
    v = np.asarray(v, dtype=np.float64)
    out = np.zeros(v.shape[:-1] + (v.shape[-1] + 1,))
    out[..., 1:] += v
    out[..., :-1] -= v
    return out


def bce_smooth(s, H, X, lam_tv, delta):
    """Smooth part of the augmented multichannel problem (Eq. 6), summed over
    the channels c that share the source s:
        f = sum_c ||h_c * s - x_c||^2 + lam_tv L_delta(D h_c) / delta
    (L_delta summed over the entries of D h_c)."""
    H = np.asarray(H, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    R = conv_full(H, np.broadcast_to(s, (H.shape[0], len(s)))) - X
    return float(np.sum(R * R)) + lam_tv / delta * float(np.sum(huber(tv_diff(H), delta)))


def bce_gradient(s, H, X, lam_tv, delta):
    """(grad_H, grad_s) of bce_smooth: with r_c = h_c * s - x_c,
        grad_{h_c} = 2 S^T r_c + (lam_tv / delta) D^T L'_delta(D h_c),
        grad_s     = sum_c 2 H_c^T r_c,
    L'_delta(z) = clip(z, -delta, delta)."""
    H = np.asarray(H, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    S = np.broadcast_to(np.asarray(s, dtype=np.float64), (H.shape[0], len(s)))
    R = conv_full(H, S) - X
    gh, gs = conv_adjoint(S, H, R)
    gh = 2.0 * gh + lam_tv / delta * tv_diff_adjoint(huber_grad(tv_diff(H), delta))
    return gh, 2.0 * gs.sum(axis=0)
