"""Multi-level 2D wavelet reconstruction W, analysis W^dagger and adjoint W^*.

Definitions (Sec. I-A, Eq. 2, Eq. 3, Eq. 4):

* zero-padded analysis of a length-M signal z with filter f (W^dagger_zpd):
      a[k] = sum_i f[i] z[2k+1-i],  k = 0..floor((M+L-1)/2)-1,  z = 0 outside [0, M)
  i.e. the full convolution z * f sampled at the odd positions;
* zero-padded synthesis S (W_zpd) onto the length-M domain, delay L':
      Y[p] = sum_k a_lo[k] g_lo[p+L'-2k-1] + a_hi[k] g_hi[p+L'-2k-1],  p = 0..M-1
  so that S Phi = I_M (perfect reconstruction of the zero-padded frame);
* with an extension E (module `extension`):
      W^dagger = W^dagger_zpd E,  W = E^dagger S,  W^* = S^T (E^dagger)^*,
  and S^T is analysis with the dual filters (the synthesis filters reversed),
  which is Eq. 4:  W^* = dual-W^dagger_zpd (E^dagger)^*.
  W W^dagger = E^dagger S Phi E = E^dagger E = I.
* 2D: separable; the level operator is the Kronecker product of the 1D
  operators along rows (axis 0) and columns (axis 1) (the paper's footnote in
  Sec. I-A says the 1D results extend "naturally" to 2D).
* "per": critically sampled circular transform (build addition),
      a[k] = sum_i f[i] y[(2k+1-i) mod N],
      y[t] = sum_k sum_m g[m] a[k] [t == (2k+1+m-L') mod N].

Two independent routes to W^* are provided so that tests can hold them
against each other and against a dense transpose:
  (i)  `wt_adjoint_transposed`: the loops of W transposed statement by
       statement (every out[i] += w*in[j] becomes in[j] += w*out[i]);
  (ii) `wt_adjoint`: the paper's formula, Eq. 4, using numpy's full
       convolution and odd-position sampling.
"""

import numpy as np

from . import extension as ext
from .filters import FilterBank, filter_bank
from .layout import band_len, level_sizes, pack, unpack

MODES = ("zero", "sym", "ppd", "per")


# ----------------------------------------------------------------- 1D along axis 0
def zpd_analysis_axis0(z: np.ndarray, f: np.ndarray) -> np.ndarray:
    """a[k] = sum_i f[i] z[2k+1-i] along axis 0 (full convolution, odd samples)."""
    M = z.shape[0]
    L = len(f)
    n = (M + L - 1) // 2
    out = np.zeros((n,) + z.shape[1:])
    for k in range(n):
        for i in range(L):
            e = 2 * k + 1 - i
            if 0 <= e < M and f[i] != 0.0:
                out[k] += f[i] * z[e]
    return out


def zpd_synthesis_axis0(a: np.ndarray, g: np.ndarray, M: int) -> np.ndarray:
    """Y[p] = sum_k a[k] g[p+L'-2k-1] for p in [0, M), scatter form."""
    L = len(g)
    Lp = L - 1
    Y = np.zeros((M,) + a.shape[1:])
    for k in range(a.shape[0]):
        for m in range(L):
            p = 2 * k + 1 + m - Lp
            if 0 <= p < M and g[m] != 0.0:
                Y[p] += g[m] * a[k]
    return Y


def per_analysis_axis0(y: np.ndarray, f: np.ndarray) -> np.ndarray:
    N = y.shape[0]
    out = np.zeros((N // 2,) + y.shape[1:])
    for k in range(N // 2):
        for i in range(len(f)):
            if f[i] != 0.0:
                out[k] += f[i] * y[(2 * k + 1 - i) % N]
    return out


def per_synthesis_axis0(a: np.ndarray, g: np.ndarray, N: int) -> np.ndarray:
    Lp = len(g) - 1
    y = np.zeros((N,) + a.shape[1:])
    for k in range(a.shape[0]):
        for m in range(len(g)):
            if g[m] != 0.0:
                y[(2 * k + 1 + m - Lp) % N] += g[m] * a[k]
    return y


def _on_axis(fn, arr, axis, *args):
    if axis == 0:
        return fn(arr, *args)
    return np.swapaxes(fn(np.swapaxes(arr, 0, 1), *args), 0, 1)


# ----------------------------------------------------------------- 1D level, one axis
def analysis_1d(y, bank: FilterBank, mode: str, kind: str, axis: int):
    """One level of 1D analysis along `axis`; returns (lo, hi).

    kind = "pinv":    W^dagger = W^dagger_zpd E      (dec filters, plain extension)
    kind = "adjoint": W^*      = S^T (E^dagger)^*    (dual filters, weighted extension)
    """
    Lp = bank.Lp
    if kind == "pinv":
        flo, fhi = bank.dec_lo, bank.dec_hi
    elif kind == "adjoint":
        flo, fhi = bank.dual_analysis()
    else:
        raise ValueError(kind)
    if mode == "per":
        return (_on_axis(per_analysis_axis0, y, axis, flo),
                _on_axis(per_analysis_axis0, y, axis, fhi))
    z = ext.apply_E(y, Lp, mode, axis) if kind == "pinv" else \
        ext.apply_E_pinv_adjoint(y, Lp, mode, axis)
    return (_on_axis(zpd_analysis_axis0, z, axis, flo),
            _on_axis(zpd_analysis_axis0, z, axis, fhi))


def synthesis_1d(lo, hi, N: int, bank: FilterBank, mode: str, axis: int):
    """One level of 1D reconstruction W = E^dagger S along `axis` (output length N)."""
    if mode == "per":
        return (_on_axis(per_synthesis_axis0, lo, axis, bank.rec_lo, N)
                + _on_axis(per_synthesis_axis0, hi, axis, bank.rec_hi, N))
    M = N + 2 * bank.Lp
    Y = (_on_axis(zpd_synthesis_axis0, lo, axis, bank.rec_lo, M)
         + _on_axis(zpd_synthesis_axis0, hi, axis, bank.rec_hi, M))
    return ext.apply_E_pinv(Y, N, bank.Lp, mode, axis)


# ----------------------------------------------------------------- 2D level
def analysis_level(Y, bank, mode, kind):
    """(LL, LH, HL, HH) of one 2D level: axis-0 analysis, then axis-1 analysis."""
    v_lo, v_hi = analysis_1d(Y, bank, mode, kind, axis=0)
    LL, HL = analysis_1d(v_lo, bank, mode, kind, axis=1)
    LH, HH = analysis_1d(v_hi, bank, mode, kind, axis=1)
    return LL, LH, HL, HH


def synthesis_level(LL, LH, HL, HH, Nr, Nc, bank, mode):
    t_lo = synthesis_1d(LL, HL, Nc, bank, mode, axis=1)   # vertical lo rows
    t_hi = synthesis_1d(LH, HH, Nc, bank, mode, axis=1)   # vertical hi rows
    return synthesis_1d(t_lo, t_hi, Nr, bank, mode, axis=0)


# ----------------------------------------------------------------- multi-level
def _bank(wavelet):
    return wavelet if isinstance(wavelet, FilterBank) else filter_bank(wavelet)


def wt_analysis(image, levels, wavelet, mode, kind="pinv"):
    """Packed coefficients of W^dagger (kind="pinv") or W^* (kind="adjoint", Eq. 4)."""
    bank = _bank(wavelet)
    LL = np.asarray(image, dtype=np.float64)
    details = []
    for _ in range(levels):
        LL, LH, HL, HH = analysis_level(LL, bank, mode, kind)
        details.append((LH, HL, HH))
    return pack(LL, details)


def wt_synth(x, rows, cols, levels, wavelet, mode):
    """W x: multi-level reconstruction of the packed coefficients x."""
    bank = _bank(wavelet)
    LL, details = unpack(np.asarray(x, dtype=np.float64), rows, cols, levels, bank.L, mode)
    sizes = level_sizes(rows, cols, levels, bank.L, mode)
    for j in range(levels, 0, -1):
        (Nr, Nc), _ = sizes[j - 1]
        LH, HL, HH = details[j - 1]
        LL = synthesis_level(LL, LH, HL, HH, Nr, Nc, bank, mode)
    return LL


def wt_pinv(image, levels, wavelet, mode):
    return wt_analysis(image, levels, wavelet, mode, kind="pinv")


def wt_adjoint(image, levels, wavelet, mode):
    """W^* by the paper's formula, Eq. 4: dual analysis after (E^dagger)^*.

    Route (ii): every 1D filtering step is numpy's full convolution sampled at
    the odd positions, independent of the loops used by `wt_synth`.
    """
    bank = _bank(wavelet)
    flo, fhi = bank.dual_analysis()

    def ana(y, f, axis):
        y = np.moveaxis(y, axis, -1)
        if mode == "per":
            N = y.shape[-1]
            Lp = bank.Lp
            # periodic: pad with a wrap-around halo of L' on the left, keep the
            # full-convolution samples that see only valid wrap data
            yp = np.concatenate([y[..., (np.arange(-Lp, 0)) % N], y], axis=-1)
            full = np.apply_along_axis(lambda v: np.convolve(v, f), -1, yp)
            out = full[..., Lp + 1:Lp + N:2]
        else:
            z = ext.apply_E_pinv_adjoint(y, bank.Lp, mode, axis=y.ndim - 1)
            full = np.apply_along_axis(lambda v: np.convolve(v, f), -1, z)
            out = full[..., 1::2]
        return np.moveaxis(out, -1, axis)

    LL = np.asarray(image, dtype=np.float64)
    details = []
    for _ in range(levels):
        v_lo, v_hi = ana(LL, flo, 0), ana(LL, fhi, 0)
        LL, HL = ana(v_lo, flo, 1), ana(v_lo, fhi, 1)
        LH, HH = ana(v_hi, flo, 1), ana(v_hi, fhi, 1)
        details.append((LH, HL, HH))
    return pack(LL, details)


# ------------------------------------------------ route (i): statement-wise transpose of W
def _synthesis_1d_T(Yout_adj, N_in_lo, bank, mode, axis):
    """Transpose of synthesis_1d: returns (lo_adj, hi_adj) given the output adjoint."""
    Lp = bank.Lp
    y = np.moveaxis(Yout_adj, axis, 0)
    N = y.shape[0]
    outs = []
    for g in (bank.rec_lo, bank.rec_hi):
        a = np.zeros((N_in_lo,) + y.shape[1:])
        if mode == "per":
            # forward: y[(2k+1+m-L') mod N] += g[m] a[k]
            for k in range(N_in_lo):
                for m in range(len(g)):
                    a[k] += g[m] * y[(2 * k + 1 + m - Lp) % N]
        else:
            # forward: out[src[p]] += Y[p] / c[src[p]];  Y[p] += g[m] a[k], p = 2k+1+m-L'
            src = ext.ext_map(N, Lp, mode)
            c = ext.copy_counts(N, Lp, mode).astype(np.float64)
            M = N + 2 * Lp
            Yadj = np.zeros((M,) + y.shape[1:])
            for p in range(M):
                if src[p] >= 0:
                    Yadj[p] += y[src[p]] / c[src[p]]
            for k in range(N_in_lo):
                for m in range(len(g)):
                    p = 2 * k + 1 + m - Lp
                    if 0 <= p < M:
                        a[k] += g[m] * Yadj[p]
        outs.append(np.moveaxis(a, 0, axis))
    return outs


def wt_adjoint_transposed(image, levels, wavelet, mode):
    """W^* as the statement-by-statement transpose of `wt_synth` (route (i))."""
    bank = _bank(wavelet)
    rows, cols = np.shape(image)
    sizes = level_sizes(rows, cols, levels, bank.L, mode)
    LLadj = np.asarray(image, dtype=np.float64)
    details = []
    for j in range(1, levels + 1):
        _, (nr, nc) = sizes[j - 1]
        # forward level: t_lo = syn1(LL,HL; axis1), t_hi = syn1(LH,HH; axis1), out = syn1(t_lo,t_hi; axis0)
        t_lo_adj, t_hi_adj = _synthesis_1d_T(LLadj, nr, bank, mode, axis=0)
        LL_adj, HL_adj = _synthesis_1d_T(t_lo_adj, nc, bank, mode, axis=1)
        LH_adj, HH_adj = _synthesis_1d_T(t_hi_adj, nc, bank, mode, axis=1)
        details.append((LH_adj, HL_adj, HH_adj))
        LLadj = LL_adj
    return pack(LLadj, details)


def dense_synth(rows, cols, levels, wavelet, mode):
    """Dense matrix of W (columns = W e_i); tiny sizes only."""
    bank = _bank(wavelet)
    from .layout import num_coeffs
    C = num_coeffs(rows, cols, levels, bank.L, mode)
    # all unit vectors at once, as a trailing batch axis
    img = wt_synth(np.eye(C), rows, cols, levels, bank, mode)
    return img.reshape(rows * cols, C)
