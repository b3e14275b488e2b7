"""Pins of the extension operators against the block matrices of Sec. I-A."""
import numpy as np
import pytest

from oracle import extension as ext


def _P(n):
    return np.eye(n)[::-1]


def _Esym_blocks(N, Lp):
    # [I P; I 0 0; 0 I_{N-2L'} 0; 0 0 I; 0 0 I P], the displayed E_sym (N > 2L')
    E = np.zeros((N + 2 * Lp, N))
    I = np.eye(Lp)
    E[0:Lp, 0:Lp] = I @ _P(Lp)
    E[Lp:2 * Lp, 0:Lp] = I
    E[2 * Lp:N, Lp:N - Lp] = np.eye(N - 2 * Lp)
    E[N:N + Lp, N - Lp:N] = I
    E[N + Lp:N + 2 * Lp, N - Lp:N] = I @ _P(Lp)
    return E


def _Eper_blocks(N, Lp):
    # [0 0 I; I_N; I 0 0], the displayed E_per
    E = np.zeros((N + 2 * Lp, N))
    E[0:Lp, N - Lp:N] = np.eye(Lp)
    E[Lp:Lp + N, :] = np.eye(N)
    E[Lp + N:, 0:Lp] = np.eye(Lp)
    return E


def _Ezpd_blocks(N, Lp):
    return np.vstack([np.zeros((Lp, N)), np.eye(N), np.zeros((Lp, N))])


@pytest.mark.parametrize("N,Lp", [(7, 3), (10, 1), (20, 9), (12, 5)])
def test_dense_E_matches_displayed_blocks(N, Lp):
    assert np.array_equal(ext.E_dense(N, Lp, "zero"), _Ezpd_blocks(N, Lp))
    assert np.array_equal(ext.E_dense(N, Lp, "sym"), _Esym_blocks(N, Lp))
    assert np.array_equal(ext.E_dense(N, Lp, "ppd"), _Eper_blocks(N, Lp))


@pytest.mark.parametrize("N,Lp", [(7, 3), (20, 9)])
def test_pinv_adjoint_half_weights_displayed(N, Lp):
    # (E_sym^dagger)^* and (E_per^dagger)^*: the same blocks with 1/2 on the 2L' boundary rows
    for mode, blocks in (("sym", _Esym_blocks), ("ppd", _Eper_blocks)):
        E = blocks(N, Lp)
        want = E.copy()
        c = E.sum(axis=0)
        assert set(np.unique(c)) == {1.0, 2.0}
        want = want / c[None, :]
        got = np.linalg.pinv(E).T
        assert np.allclose(got, want, atol=1e-13)
        # and the oracle's weighted extension applies exactly this matrix
        Y = np.eye(N)
        assert np.allclose(ext.apply_E_pinv_adjoint(Y, Lp, mode, axis=0), want, atol=1e-15)


@pytest.mark.parametrize("mode", ext.MODES)
@pytest.mark.parametrize("N", list(range(1, 14)))
@pytest.mark.parametrize("Lp", [1, 3, 9])
def test_pinv_and_its_adjoint_all_sizes(mode, N, Lp):
    """1/c weights equal numpy's pseudoinverse for every N, including N <= 2L'
    (where the paper says some 1/2 become 1/3)."""
    E = ext.E_dense(N, Lp, mode)
    Y = np.eye(N)
    Epinv_adj = ext.apply_E_pinv_adjoint(Y, Lp, mode, axis=0)
    Epinv = ext.apply_E_pinv(np.eye(N + 2 * Lp), N, Lp, mode, axis=0)
    pinv = np.linalg.pinv(E)
    assert np.allclose(Epinv, pinv, atol=1e-13)
    assert np.allclose(Epinv_adj, pinv.T, atol=1e-13)
    assert np.allclose(Epinv @ E, np.eye(N), atol=1e-14)      # E^dagger E = I
    if mode == "zero":                                          # orthonormal columns
        assert np.array_equal(E.T @ E, np.eye(N))


def test_one_third_weights_appear():
    # N <= 2L' gives copy counts of 3 (the 1/3 entries mentioned in Sec. I-A)
    assert 3 in ext.copy_counts(4, 3, "sym")
    assert 3 in ext.copy_counts(4, 3, "ppd")
    assert max(ext.copy_counts(7, 3, "sym")) == 2


@pytest.mark.parametrize("N", list(range(1, 14)))
@pytest.mark.parametrize("Lp", [1, 3, 8, 9, 16, 31])
def test_ext_map_matches_numpy_pad(N, Lp):
    """The index maps against numpy's own padding of arange(N): half-point
    symmetric ('symmetric', which repeats the reflection when the pad is wider
    than the signal), periodic ('wrap') and zero ('constant').  This pins the
    repeated-reflection branch used for L' >= N (Sec. I-A, reading C1) to a
    source that shares nothing with the oracle."""
    idx = np.arange(N)
    assert np.array_equal(ext.ext_map(N, Lp, "sym"), np.pad(idx, Lp, mode="symmetric"))
    assert np.array_equal(ext.ext_map(N, Lp, "ppd"), np.pad(idx, Lp, mode="wrap"))
    assert np.array_equal(ext.ext_map(N, Lp, "zero"), np.pad(idx, Lp, mode="constant", constant_values=-1))


# Half-point symmetric extension by L' = 3 of [a], [a b], [a b c], written out by
# hand: the signal mirrored about each end, the mirror image mirrored again.
_SYM_TABLE_LP3 = {
    1: "a a a | a | a a a",
    2: "b b a | a b | b a a",
    3: "c b a | a b c | c b a",
}


@pytest.mark.parametrize("N", [1, 2, 3])
def test_ext_map_sym_hand_table(N):
    want = [ord(ch) - ord("a") for ch in _SYM_TABLE_LP3[N].split() if ch != "|"]
    assert ext.ext_map(N, 3, "sym").tolist() == want


def test_ext_map_sym_whole_point_would_fail():
    """A whole-point reflection (y[-1] = y[1]) or an off-by-one in the repeated
    branch changes the map at N = 2, L' = 9 (so the pins above would catch it)."""
    N, Lp = 2, 9
    got = ext.ext_map(N, Lp, "sym")
    whole = np.pad(np.arange(N), Lp, mode="reflect")
    assert not np.array_equal(got, whole)
    shifted = np.pad(np.arange(N), (Lp - 1, Lp + 1), mode="symmetric")
    assert not np.array_equal(got, shifted)
