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
