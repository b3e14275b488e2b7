"""Band sizes and the packed (logical, unpadded) coefficient order.

Per level and per axis (readings of Sec. I-A, where the paper writes
W^dagger = W^dagger_zpd E and leaves the transform's length implicit):

* zero / sym / ppd: the level input of length N is extended to M = N + 2L';
  W^dagger_zpd is the full zero-padded analysis of that length-M signal (full
  convolution, M + L - 1 = N + 3L' outputs) keeping the odd 0-based positions,
  so each band has n = floor((N + 3L') / 2) samples.
* per (critically sampled circular transform, a build addition that makes
  W^* = W^-1 for orthogonal filters): n = N / 2, N even at every level.

Packed order: [LL_J, (LH_J, HL_J, HH_J), ..., (LH_1, HL_1, HH_1)], each band
row-major.  A band is named by its (vertical, horizontal) filters:
LH = (hi, lo), HL = (lo, hi), HH = (hi, hi).
"""

BANDS = ("LH", "HL", "HH")
BAND_FILTERS = {"LL": (0, 0), "LH": (1, 0), "HL": (0, 1), "HH": (1, 1)}  # 0 = lo, 1 = hi


def band_len(N: int, L: int, mode: str) -> int:
    if mode == "per":
        if N % 2:
            raise ValueError("per mode needs an even length at every level")
        return N // 2
    return (N + 3 * (L - 1)) // 2


def level_sizes(rows: int, cols: int, levels: int, L: int, mode: str):
    """[(N_r, N_c) of LL_{j-1}, (n_r, n_c) of the level-j bands] for j = 1..J."""
    out = []
    Nr, Nc = rows, cols
    for _ in range(levels):
        nr, nc = band_len(Nr, L, mode), band_len(Nc, L, mode)
        out.append(((Nr, Nc), (nr, nc)))
        Nr, Nc = nr, nc
    return out


def num_coeffs(rows, cols, levels, L, mode) -> int:
    sizes = level_sizes(rows, cols, levels, L, mode)
    total = 0
    for _, (nr, nc) in sizes:
        total += 3 * nr * nc
    nr, nc = sizes[-1][1]
    return total + nr * nc


def pack(LL, details):
    """details[j-1] = (LH_j, HL_j, HH_j); returns the packed vector (bands may
    carry trailing batch axes, which are kept)."""
    import numpy as np

    def flat(b):
        return b.reshape((b.shape[0] * b.shape[1],) + b.shape[2:])
    parts = [flat(LL)]
    for j in range(len(details), 0, -1):
        parts += [flat(b) for b in details[j - 1]]
    return np.concatenate(parts, axis=0)


def unpack(x, rows, cols, levels, L, mode):
    import numpy as np
    sizes = level_sizes(rows, cols, levels, L, mode)
    pos = 0
    nr, nc = sizes[-1][1]
    x = np.asarray(x)
    tail = x.shape[1:]
    LL = x[pos:pos + nr * nc].reshape((nr, nc) + tail)
    pos += nr * nc
    details = [None] * levels
    for j in range(levels, 0, -1):
        nr, nc = sizes[j - 1][1]
        bands = []
        for _ in range(3):
            bands.append(x[pos:pos + nr * nc].reshape((nr, nc) + tail))
            pos += nr * nc
        details[j - 1] = tuple(bands)
    assert pos == x.shape[0]
    return LL, details
