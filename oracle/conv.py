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
