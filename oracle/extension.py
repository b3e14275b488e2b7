"""Signal-extension operators of Sec. I-A, as index maps and as dense matrices.

A 1D signal y[0..N-1] is extended by L' = L - 1 samples on each side to the
length M = N + 2L' (Sec. I-A).  Position p of the extended signal holds
y[ext(p - L')], or zero where the extension is zero-padded.  The extension
modes:

* "zero": zero-padded extension E_zpd (the first displayed matrix of Sec. I-A);
* "sym":  half-point symmetric extension E_sym.  The printed index line of the
          left/right extension is garbled (it lists L samples on the left and
          indexes past the signal on the right); read as L' samples per side,
          left = y[L'-1..0], right = y[N-1..N-L'], which is what the block
          matrix with I_{L'}P blocks encodes.  For L' >= N the reflection
          repeats (index mod 2N, mirrored).
* "ppd":  the periodic extension E_per of Sec. I-A (left = the last L'
          samples, right = the first L'); redundant, so W is not square.

E has one 1 in every row, hence E^T E = diag(c) with c[j] the number of
extended positions holding y[j]; E^dagger = diag(1/c) E^T and
(E^dagger)^* = E diag(1/c).  With N > 2L' this reproduces the 1/2 entries of
the displayed (E_sym^dagger)^* and (E_per^dagger)^*; for N <= 2L' it gives the
1/3 entries the paper mentions.
"""

import numpy as np

MODES = ("zero", "sym", "ppd")


def ext_index(x: int, N: int, mode: str):
    """Source index of virtual position x (image coordinates), None for a zero."""
    if mode == "zero":
        return x if 0 <= x < N else None
    if mode == "sym":
        m = x % (2 * N)
        return m if m < N else 2 * N - 1 - m
    if mode in ("ppd", "per"):
        return x % N
    raise ValueError(mode)


def ext_map(N: int, Lp: int, mode: str):
    """src[p] for p in [0, N + 2L'): the source index of extended sample p (-1 = zero)."""
    M = N + 2 * Lp
    src = np.full(M, -1, dtype=np.int64)
    for p in range(M):
        j = ext_index(p - Lp, N, mode)
        if j is not None:
            src[p] = j
    return src


def copy_counts(N: int, Lp: int, mode: str) -> np.ndarray:
    """c[j] = number of rows of E equal to e_j (E^T E = diag(c))."""
    src = ext_map(N, Lp, mode)
    c = np.zeros(N, dtype=np.int64)
    for j in src:
        if j >= 0:
            c[j] += 1
    return c


def E_dense(N: int, Lp: int, mode: str) -> np.ndarray:
    src = ext_map(N, Lp, mode)
    E = np.zeros((len(src), N))
    for p, j in enumerate(src):
        if j >= 0:
            E[p, j] = 1.0
    return E


def apply_E(y: np.ndarray, Lp: int, mode: str, axis: int = 0) -> np.ndarray:
    """E y along `axis`: gather y at the extension map (zeros where src = -1)."""
    N = y.shape[axis]
    src = ext_map(N, Lp, mode)
    y = np.moveaxis(y, axis, 0)
    out = np.zeros((len(src),) + y.shape[1:])
    ok = src >= 0
    out[ok] = y[src[ok]]
    return np.moveaxis(out, 0, axis)


def apply_E_pinv_adjoint(y: np.ndarray, Lp: int, mode: str, axis: int = 0) -> np.ndarray:
    """(E^dagger)^* y = E diag(1/c) y along `axis` (the weighted extension)."""
    N = y.shape[axis]
    c = copy_counts(N, Lp, mode).astype(np.float64)
    shape = [1] * y.ndim
    shape[axis] = N
    return apply_E(y / c.reshape(shape), Lp, mode, axis)


def apply_E_pinv(Y: np.ndarray, N: int, Lp: int, mode: str, axis: int = 0) -> np.ndarray:
    """E^dagger Y = diag(1/c) E^T Y along `axis`: average the copies of each sample."""
    src = ext_map(N, Lp, mode)
    c = copy_counts(N, Lp, mode).astype(np.float64)
    Y = np.moveaxis(Y, axis, 0)
    out = np.zeros((N,) + Y.shape[1:])
    for p, j in enumerate(src):
        if j >= 0:
            out[j] += Y[p]
    shape = [N] + [1] * (Y.ndim - 1)
    out /= c.reshape(shape)
    return np.moveaxis(out, 0, axis)
