"""Blur operator R and its adjoint R^* (Sec. I; the gradient displayed after Eq. 1).

The paper's R is a Gaussian point-spread function applied under symmetric
(reflexive) boundary conditions and evaluated with FFTs; the operator itself
is a 2D convolution of the boundary-extended image.  Here, for a PSF of odd
length k = 2r + 1 per axis (separable: p2d = outer(p_rows, p_cols)):

    R u = C_valid(E_r u):   (R u)[i] = sum_a p[a] u[ext(i + r - a)]      (1D)
    R^* v = E_r^T C_valid^T v:
        w[x] = sum_a p[a] v0[x - r + a],  x in [-r, N + r - 1]   (v0 = 0 outside)
        (R^* v)[j] = sum_{x : ext(x) = j} w[x]                   (fold = E_r^T)

with ext the zero / half-point symmetric / circular extension by r samples.
Note the fold is E^T, not (E^dagger)^*: R contains E itself, not E^dagger.
2D applies the 1D operator along axis 0 and axis 1 (Kronecker product; the
boundary extensions are separable).
"""

import numpy as np

from .extension import ext_index

BCS = ("zero", "sym", "per")


def gaussian_psf(k: int, sigma: float) -> np.ndarray:
    """k_i = exp(-(i-c)^2 / (2 sigma^2)), c = (k-1)/2, normalised to sum 1."""
    c = (k - 1) / 2.0
    i = np.arange(k, dtype=np.float64)
    p = np.exp(-((i - c) ** 2) / (2.0 * sigma * sigma))
    return p / p.sum()


def gaussian_psf_dsigma(k: int, sigma: float) -> np.ndarray:
    """d/dsigma of gaussian_psf(k, sigma): with q_i the normalised taps and
    d_i = i - c, dq_i/dsigma = q_i (d_i^2 - sum_j q_j d_j^2) / sigma^3
    (quotient rule on e_i / sum e, de_i/dsigma = e_i d_i^2 / sigma^3).  The
    separable PSF q (x) q then has derivative q' (x) q + q (x) q'; R is
    linear in its taps, so dR/dsigma u = blur(u, q', q) + blur(u, q, q')."""
    q = gaussian_psf(k, sigma)
    c = (k - 1) / 2.0
    d2 = (np.arange(k, dtype=np.float64) - c) ** 2
    return q * (d2 - float(np.sum(q * d2))) / sigma ** 3


def _bc(bc):
    return "sym" if bc == "sym" else ("per" if bc == "per" else "zero")


def blur_1d_axis0(u: np.ndarray, p: np.ndarray, bc: str) -> np.ndarray:
    k = len(p)
    assert k % 2 == 1
    r = k // 2
    N = u.shape[0]
    out = np.zeros_like(u, dtype=np.float64)
    for i in range(N):
        for a in range(k):
            j = ext_index(i + r - a, N, _bc(bc))
            if j is not None:
                out[i] += p[a] * u[j]
    return out


def blur_adjoint_1d_axis0(v: np.ndarray, p: np.ndarray, bc: str) -> np.ndarray:
    k = len(p)
    r = k // 2
    N = v.shape[0]
    g = np.zeros_like(v, dtype=np.float64)
    for x in range(-r, N + r):
        w = np.zeros(v.shape[1:])
        for a in range(k):
            i = x - r + a
            if 0 <= i < N:
                w = w + p[a] * v[i]
        j = ext_index(x, N, _bc(bc))
        if j is not None:
            g[j] += w
    return g


def _axes(fn, img, p_rows, p_cols, bc):
    img = np.asarray(img, dtype=np.float64)
    t = fn(img, np.asarray(p_rows, dtype=np.float64), bc)
    return np.swapaxes(fn(np.swapaxes(t, 0, 1), np.asarray(p_cols, dtype=np.float64), bc), 0, 1)


def blur(u, p_rows, p_cols, bc):
    """R u for the separable PSF outer(p_rows, p_cols)."""
    return _axes(blur_1d_axis0, u, p_rows, p_cols, bc)


def blur_adjoint(v, p_rows, p_cols, bc):
    """R^* v (correlation over the extended domain, then fold with E^T)."""
    return _axes(blur_adjoint_1d_axis0, v, p_rows, p_cols, bc)


def blur_normal(u, b, p_rows, p_cols, bc):
    """(R^*(R u - b), 1/2 ||R u - b||^2): the data-term gradient in image space."""
    res = blur(u, p_rows, p_cols, bc) - np.asarray(b, dtype=np.float64)
    return blur_adjoint(res, p_rows, p_cols, bc), 0.5 * float(np.sum(res * res))


def dense_blur(rows, cols, p_rows, p_cols, bc):
    Rm = np.zeros((rows * cols, rows * cols))
    for i in range(rows * cols):
        e = np.zeros(rows * cols)
        e[i] = 1.0
        Rm[:, i] = blur(e.reshape(rows, cols), p_rows, p_cols, bc).ravel()
    return Rm
