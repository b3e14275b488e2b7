"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

Holds none of the method's arithmetic (no wavelet, blur or convolution): it only
draws numbers.  The paper's own data (a resolution test chart, simulated
underwater-acoustic recordings) is not available; these generators stand in
with the same structure:

* `piecewise_smooth_image`: a linear ramp (alpha*i + beta*j) rescaled to
  [0, 0.5], plus 12 axis-aligned rectangles and 12 ellipses each adding a
  uniform value in [-0.5, 0.5] inside, clipped to [0, 1] (a stand-in for the
  resolution chart of Sec. I-B);
* `gaussian_noise`: N(0, std^2) with std = 1e-3 by default (the blurred image
  is b = R img + noise; "small amount of Gaussian noise" in Sec. I-B);
* `channel_problem`: batch rows of N(0,1) source signals of length N and
  K-tap channels h[k] = z_k exp(-k / (K/4)), z ~ N(0,1) (the exponentially
  decaying channels of Sec. II), plus a perturbed estimate (h_est, s_est) at
  which gradients are taken, and observation noise of std 0.005 (Sec. II);
* `random_vector`: N(0,1) start vectors (power iteration) and test vectors.
* `he_normal_params`: initial weights of a stack of 3x3 convolution layers,
  N(0, 2 / (9 Cin)) per weight (He et al.'s fan-in scaling for ReLU), the last
  layer scaled by `last_scale`, biases 0, concatenated layer by layer as
  (weights in (Cout, Cin, 3, 3) order, then Cout biases).

Every draw uses numpy's PCG64 generator seeded by the caller.
"""

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(seed))


def piecewise_smooth_image(rows: int, cols: int, seed: int, shapes: int = 12) -> np.ndarray:
    g = rng(seed)
    i = np.arange(rows, dtype=np.float64)[:, None]
    j = np.arange(cols, dtype=np.float64)[None, :]
    alpha, beta = g.uniform(-1.0, 1.0, size=2)
    ramp = alpha * i / max(rows - 1, 1) + beta * j / max(cols - 1, 1)
    ramp = ramp - ramp.min()
    if ramp.max() > 0:
        ramp = 0.5 * ramp / ramp.max()
    img = ramp.copy()
    for _ in range(shapes):                      # rectangles
        r0, r1 = np.sort(g.integers(0, rows + 1, size=2))
        c0, c1 = np.sort(g.integers(0, cols + 1, size=2))
        img[r0:r1, c0:c1] += g.uniform(-0.5, 0.5)
    for _ in range(shapes):                      # ellipses
        ci, cj = g.uniform(0, rows), g.uniform(0, cols)
        ai, aj = g.uniform(0.03, 0.3) * rows, g.uniform(0.03, 0.3) * cols
        inside = ((i - ci) / ai) ** 2 + ((j - cj) / aj) ** 2 <= 1.0
        img[inside] += g.uniform(-0.5, 0.5)
    return np.clip(img, 0.0, 1.0)


def gaussian_noise(shape, seed: int, std: float = 1e-3) -> np.ndarray:
    return rng(seed).normal(0.0, std, size=shape)


def random_vector(shape, seed: int) -> np.ndarray:
    return rng(seed).standard_normal(size=shape)


def random_taps(k: int, seed: int, normalise: bool = True) -> np.ndarray:
    """Positive asymmetric taps (test PSFs for which R^* != R)."""
    t = rng(seed).uniform(0.05, 1.0, size=k)
    return t / t.sum() if normalise else t


def channel_problem(batch: int, n: int, k: int, seed: int, noise_std: float = 0.005,
                    perturb: float = 0.1):
    """Returns dict(s, h, x, s_est, h_est) for the blind-channel gradient."""
    g = rng(seed)
    s = g.standard_normal((batch, n))
    tau = k / 4.0
    h = g.standard_normal((batch, k)) * np.exp(-np.arange(k) / tau)[None, :]
    s_est = s + perturb * g.standard_normal((batch, n))
    h_est = h + perturb * g.standard_normal((batch, k)) * np.exp(-np.arange(k) / tau)[None, :]
    noise = noise_std * g.standard_normal((batch, n + k - 1))
    return {"s": s, "h": h, "noise": noise, "s_est": s_est, "h_est": h_est}


def he_normal_params(shapes, seed: int, last_scale: float = 0.1) -> np.ndarray:
    """Flat initial parameters for 3x3 layers of (Cout, Cin) `shapes`."""
    g = rng(seed)
    parts = []
    for i, (co, ci) in enumerate(shapes):
        w = g.standard_normal(co * ci * 9) * np.sqrt(2.0 / (9 * ci))
        if i == len(shapes) - 1:
            w *= last_scale
        parts += [w, np.zeros(co)]
    return np.concatenate(parts)
