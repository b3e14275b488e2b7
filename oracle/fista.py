"""Synthesis-formulation deblurring (Eq. 1) solved by FISTA (Sec. I-B).

    min_x  F(x) = 1/2 ||R W x - b||^2 + lambda ||x||_1,
    grad f(x) = W^* R^* (R W x - b)                 (the display after Eq. 1)

FISTA (Beck & Teboulle, cited for the experiments of Sec. I-B; the paper
prints none of its constants, so these are readings):
    x_0 = 0, y_1 = x_0, t_1 = 1, constant step 1/L_f;
    x_k     = soft(y_k - grad f(y_k) / L_f, lambda / L_f)
    t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
    y_{k+1} = x_k + ((t_k - 1) / t_{k+1}) (x_k - x_{k-1})
    soft(v, tau) = sign(v) max(|v| - tau, 0)   (|v| <= tau gives 0)
lambda applies to every coefficient, the coarse LL band included.
L_f = 1.01 * (power-iteration estimate of ||W^* R^* R W||), the estimate being
||A^* A v|| after `iters` normalised iterations from a caller-supplied start.

Problem(gradient="pinv") is the variant the paper argues against (Sec. I-A,
the W^dagger vs W^* discussion of Sec. I-B, I-C): the analysis operator
W^dagger stands in for W^* in grad f, so the iteration no longer follows the
gradient of F unless W^dagger = W^* (orthogonal filters, periodic boundary).
"""

from dataclasses import dataclass

import numpy as np

from . import blur as _blur
from . import wavelet as _wt


@dataclass
class Problem:
    rows: int
    cols: int
    levels: int
    wavelet: str
    mode: str          # wavelet extension: zero / sym / ppd / per
    p_rows: np.ndarray
    p_cols: np.ndarray
    blur_bc: str       # zero / sym / per
    b: np.ndarray
    lam: float
    gradient: str = "adjoint"  # "adjoint": W^*;  "pinv": W^dagger in its place

    def A(self, x):
        u = _wt.wt_synth(x, self.rows, self.cols, self.levels, self.wavelet, self.mode)
        return _blur.blur(u, self.p_rows, self.p_cols, self.blur_bc)

    def At(self, v):
        """The operator used in grad f: A^* = W^* R^*, or W^dagger R^* for gradient="pinv"."""
        g = _blur.blur_adjoint(v, self.p_rows, self.p_cols, self.blur_bc)
        if self.gradient == "pinv":
            return _wt.wt_pinv(g, self.levels, self.wavelet, self.mode)
        return _wt.wt_adjoint(g, self.levels, self.wavelet, self.mode)

    def At_exact(self, v):
        g = _blur.blur_adjoint(v, self.p_rows, self.p_cols, self.blur_bc)
        return _wt.wt_adjoint(g, self.levels, self.wavelet, self.mode)

    def grad(self, x):
        """(grad f(x), f(x))."""
        res = self.A(x) - self.b
        return self.At(res), 0.5 * float(np.sum(res * res))

    def objective(self, x):
        res = self.A(x) - self.b
        return 0.5 * float(np.sum(res * res)) + self.lam * float(np.sum(np.abs(x)))


def soft(v, tau):
    return np.sign(v) * np.maximum(np.abs(v) - tau, 0.0)


def t_next(t):
    return (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0


def power_iteration(prob: Problem, v0, iters=50):
    """Estimate of the largest eigenvalue of A^* A (A = R W) by `iters` steps."""
    v = np.asarray(v0, dtype=np.float64)
    v = v / np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = prob.At_exact(prob.A(v))
        lam = float(np.linalg.norm(w))
        v = w / lam
    return lam


def lipschitz(prob: Problem, v0, iters=50):
    return 1.01 * power_iteration(prob, v0, iters)


def fista_step(prob: Problem, x_prev, y, t, L):
    """One iteration: returns (x_k, y_{k+1}, t_{k+1}) from (x_{k-1}, y_k, t_k)."""
    g, _ = prob.grad(y)
    x = soft(y - g / L, prob.lam / L)
    t1 = t_next(t)
    y1 = x + ((t - 1.0) / t1) * (x - x_prev)
    return x, y1, t1


def fista(prob: Problem, L, iters, record_every=0, x0=None):
    """Run `iters` FISTA iterations; returns (x, [(k, F(x_k)), ...])."""
    from .layout import num_coeffs
    from .filters import filter_bank
    C = num_coeffs(prob.rows, prob.cols, prob.levels, filter_bank(prob.wavelet).L, prob.mode)
    x = np.zeros(C) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    y = x.copy()
    t = 1.0
    hist = []
    for k in range(1, iters + 1):
        x, y, t = fista_step(prob, x, y, t, L)
        if record_every and (k % record_every == 0 or k == iters):
            hist.append((k, prob.objective(x)))
    return x, hist
