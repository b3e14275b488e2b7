"""Unrolled FISTA and its reverse-mode derivative (float64) - test infrastructure.

Differentiating through the deblurring solve of Eq. 1 (Sec. I) with the
chain rule the paper states for the adjoint (grad of l(A x) is A^* grad l):
the backward of an iteration applies A = R W and A^* = W^* R^* themselves,
which is only correct with the exact adjoint W^* (Eq. 4).

Iteration (0-based, the GPU library's order; the same iterates as
oracle.fista.fista_step):  x_0 = y_0 = 0, t_0 = 1,
    z_k     = y_k - (1/L) A^*(A y_k - b)
    x_{k+1} = soft(z_k, lam / L)
    t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2,  beta_k = (t_k - 1) / t_{k+1}
    y_{k+1} = x_{k+1} + beta_k (x_{k+1} - x_k)
Loss after N steps:  l = 1/2 ||W x_N - u_ref||^2  (W: synthesis, Eq. 2).
L is a constant of the unrolled map (not differentiated).  The PSF is the
separable Gaussian q (x) q of width sigma (blur.gaussian_psf).

Reverse mode, k = N-1 .. 0, with Xp_{k+1} the adjoint of x_{k+1} collected
so far and Y_{k+1} that of y_{k+1} (Xp_N = W^*(W x_N - u_ref), Y_N = 0):
    X       = Xp_{k+1} + (1 + beta_k) Y_{k+1}
    zbar    = X [x_{k+1} != 0]                 (soft' = 1 where |z| > tau, else 0)
    dl/dtau += -sum sign(x_{k+1}) X            (d soft / d tau = -sign(z) there)
    u = W zbar
    Y_k     = zbar - (1/L) W^* R^* R u
    Xp_k    = -beta_k Y_{k+1}
    dl/db  += (1/L) R u
    dl/dsigma += -(1/L) (<R' u, A y_k - b> + <R u, R' W y_k>),  R' = dR/dsigma
and dl/dlam = (dl/dtau) / L.  Pinned against central differences of
`unrolled_loss` (tests/test_oracle_unrolled.py).
"""

import numpy as np

from . import blur as _blur
from . import wavelet as _wt
from .fista import soft, t_next


class Setup:
    """The problem data of one unrolled solve (float64)."""

    def __init__(self, rows, cols, levels, wavelet, mode, k, sigma, blur_bc, b, lam, L):
        self.rows, self.cols, self.levels, self.wavelet, self.mode = rows, cols, levels, wavelet, mode
        self.k, self.sigma, self.blur_bc = k, float(sigma), blur_bc
        self.b = np.asarray(b, dtype=np.float64)
        self.lam, self.L = float(lam), float(L)
        self.q = _blur.gaussian_psf(k, sigma)
        self.dq = _blur.gaussian_psf_dsigma(k, sigma)

    def W(self, x):
        return _wt.wt_synth(x, self.rows, self.cols, self.levels, self.wavelet, self.mode)

    def Wt(self, img):
        return _wt.wt_adjoint(img, self.levels, self.wavelet, self.mode)

    def R(self, u):
        return _blur.blur(u, self.q, self.q, self.blur_bc)

    def Rt(self, v):
        return _blur.blur_adjoint(v, self.q, self.q, self.blur_bc)

    def dR(self, u):
        """dR/dsigma u = R[q', q] u + R[q, q'] u."""
        return _blur.blur(u, self.dq, self.q, self.blur_bc) + _blur.blur(u, self.q, self.dq, self.blur_bc)


def forward(S: Setup, n_steps: int, ncoef: int):
    """All iterates: xs[k], ys[k] for k = 0..n_steps and the betas."""
    x = np.zeros(ncoef)
    y = np.zeros(ncoef)
    t = 1.0
    xs, ys, betas = [x], [y], []
    for _ in range(n_steps):
        z = y - S.Wt(S.Rt(S.R(S.W(y)) - S.b)) / S.L
        x1 = soft(z, S.lam / S.L)
        t1 = t_next(t)
        beta = (t - 1.0) / t1
        y = x1 + beta * (x1 - x)
        x, t = x1, t1
        xs.append(x)
        ys.append(y)
        betas.append(beta)
    return xs, ys, betas


def unrolled_loss(S: Setup, n_steps: int, u_ref, ncoef: int) -> float:
    xs, _, _ = forward(S, n_steps, ncoef)
    e = S.W(xs[-1]) - u_ref
    return 0.5 * float(np.sum(e * e))


def unrolled_grads(S: Setup, n_steps: int, u_ref, ncoef: int):
    """(loss, dl/dlam, dl/dsigma, dl/db) by the reverse recursion above."""
    xs, ys, betas = forward(S, n_steps, ncoef)
    e = S.W(xs[-1]) - u_ref
    loss = 0.5 * float(np.sum(e * e))
    Xp = S.Wt(e)
    Y = np.zeros(ncoef)
    dtau = 0.0
    dsigma = 0.0
    db = np.zeros_like(S.b)
    for k in range(n_steps - 1, -1, -1):
        beta = betas[k]
        X = Xp + (1.0 + beta) * Y
        on = xs[k + 1] != 0.0
        zbar = np.where(on, X, 0.0)
        dtau += -float(np.sum(np.sign(xs[k + 1]) * X))
        u = S.W(zbar)
        Ru = S.R(u)
        Y_k = zbar - S.Wt(S.Rt(Ru)) / S.L
        Xp = -beta * Y
        db += Ru / S.L
        Wy = S.W(ys[k])
        r = S.R(Wy) - S.b
        dsigma += -(float(np.sum(S.dR(u) * r)) + float(np.sum(Ru * S.dR(Wy)))) / S.L
        Y = Y_k
    return loss, dtau / S.L, dsigma, db
