"""Parity of the CUDA FISTA step, objective and step size with the float64 oracle (Eq. 1)."""
import numpy as np
import pytest
import torch

from oracle import blur as oblur
from oracle import fista as ofista
from oracle import wavelet as owt
from synthetic_inputs import gaussian_noise, piecewise_smooth_image, random_vector
from tests.gpu_util import assert_close, image_dev, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def adj():
    import paper_1707_02018_gb300 as adj
    adj.lib()
    return adj


def _setup(adj, rows, cols, J, w, mode, k, sigma, lam, seed, bc=None):
    bc = bc or mode
    p = oblur.gaussian_psf(k, sigma) if k > 1 else np.array([1.0])
    img = piecewise_smooth_image(rows, cols, seed)
    b = oblur.blur(img, p, p, bc) + gaussian_noise((rows, cols), seed + 1)
    prob = ofista.Problem(rows, cols, J, w, mode, p, p, bc, b, lam)
    wt = adj.WtPlan(rows, cols, J, w, mode)
    bl = adj.BlurPlan(rows, cols, p, p, bc)
    db = image_dev(wt, b)
    return prob, wt, bl, db


def test_lipschitz_matches_oracle(adj):
    prob, wt, bl, db = _setup(adj, 256, 256, 3, "db2", "sym", 9, 1.5, 1e-3, 1)
    v0 = random_vector(wt.logical_size, 77)
    L_or = ofista.lipschitz(prob, v0, iters=50)
    f = adj.Fista(wt, bl, db, 1e-3)
    L_gpu = f.lipschitz(wt.pack(v0), iters=50)
    assert abs(L_gpu - L_or) <= 1e-5 * L_or


def test_fista_trajectory_256(adj):
    """256^2, db2 J=3, symmetric BC, 9x9 sigma=1.5, lambda=1e-3, 100 iterations:
    objective within 1e-5 relative at every 10th iteration, iterate within 1e-4."""
    prob, wt, bl, db = _setup(adj, 256, 256, 3, "db2", "sym", 9, 1.5, 1e-3, 1)
    L = ofista.lipschitz(prob, random_vector(wt.logical_size, 77), iters=50)
    f = adj.Fista(wt, bl, db, 1e-3, L)
    x, y, t = np.zeros(wt.logical_size), np.zeros(wt.logical_size), 1.0
    for k in range(1, 101):
        x, y, t = ofista.fista_step(prob, x, y, t, L)
        if k % 10 == 0:
            Fg = f.step(objective=True)
            Fo = prob.objective(x)
            assert abs(Fg - Fo) <= 1e-5 * Fo, (k, Fg, Fo)
        else:
            f.step()
    assert abs(f.state.t - t) < 1e-12 * t and f.state.k == 100
    xg = wt.unpack(f.x).cpu().numpy()
    assert rel_err(xg, x) <= 1e-4
    assert rel_err(wt.unpack(f.y).cpu().numpy(), y) <= 1e-4


@pytest.mark.parametrize("mode", ["per", "zero", "ppd"])
def test_fista_steps_other_boundaries(adj, mode):
    bc = "per" if mode in ("per", "ppd") else "zero"
    prob, wt, bl, db = _setup(adj, 96, 64, 3, "cdf97", mode, 7, 1.2, 2e-3, 5, bc=bc)
    L = ofista.lipschitz(prob, random_vector(wt.logical_size, 3), iters=30)
    f = adj.Fista(wt, bl, db, 2e-3, L)
    x, y, t = np.zeros(wt.logical_size), np.zeros(wt.logical_size), 1.0
    for k in range(1, 21):
        x, y, t = ofista.fista_step(prob, x, y, t, L)
        Fg = f.step(objective=(k % 5 == 0))
        if k % 5 == 0:
            assert abs(Fg - prob.objective(x)) <= 1e-5 * prob.objective(x)
    assert rel_err(wt.unpack(f.x).cpu().numpy(), x) <= 1e-4


@pytest.mark.parametrize("mode", ["sym", "zero", "per", "ppd"])
@pytest.mark.parametrize("tiled_only", [False, True])
def test_fista_steps_large_levels(adj, mode, tiled_only):
    """1600 x 1664, db4 J=2: level 1 runs the prox in the persistent TMA
    analysis kernel (with the tiled kernel on the border tiles unless the TMA
    tiles cover the level), or, switched off, in the tiled kernel alone."""
    bc = "per" if mode in ("per", "ppd") else mode
    prob, wt, bl, db = _setup(adj, 1600, 1664, 2, "db4", mode, 9, 1.5, 1e-3, 21, bc=bc)
    if tiled_only:
        for op in ("synth", "prox"):
            for j in (1, 2):
                wt.set_tma(op, j, False)
    L = 1.01  # a few steps at a fixed step size: parity does not need the estimated L_f
    f = adj.Fista(wt, bl, db, 1e-3, L)
    x, y, t = np.zeros(wt.logical_size), np.zeros(wt.logical_size), 1.0
    for k in range(1, 5):
        x, y, t = ofista.fista_step(prob, x, y, t, L)
        Fg = f.step(objective=(k % 2 == 0))
        if k % 2 == 0:
            assert abs(Fg - prob.objective(x)) <= 1e-5 * prob.objective(x)
    assert rel_err(wt.unpack(f.x).cpu().numpy(), x) <= 1e-4
    assert rel_err(wt.unpack(f.y).cpu().numpy(), y) <= 1e-4
    assert adj.device_status() == 0


def test_identity_blur_closed_form(adj):
    """R = I, circular db2: one step with L_f = 1 lands on soft(W^T b, lambda)."""
    rows = cols = 32
    lam = 0.05
    b = piecewise_smooth_image(rows, cols, 4) + gaussian_noise((rows, cols), 5, std=0.05)
    wt = adj.WtPlan(rows, cols, 3, "db2", "per")
    bl = adj.BlurPlan(rows, cols, [1.0], [1.0], "per")
    f = adj.Fista(wt, bl, image_dev(wt, b), lam, 1.0)
    f.step()
    want = ofista.soft(owt.wt_adjoint(b, 3, "db2", "per"), lam)
    assert_close(wt.unpack(f.x).cpu().numpy(), want, abs_max=5e-5, what="closed form")
    assert np.mean(want == 0) > 0.1
    f.step()
    assert_close(wt.unpack(f.x).cpu().numpy(), want, abs_max=5e-5, what="stays")


def test_objective_api(adj):
    prob, wt, bl, db = _setup(adj, 128, 96, 2, "db4", "sym", 5, 1.0, 3e-3, 8)
    f = adj.Fista(wt, bl, db, 3e-3, 1.0)
    x = random_vector(wt.logical_size, 6)
    Fg = f.objective(wt.pack(x))
    assert abs(Fg - prob.objective(x)) <= 1e-5 * prob.objective(x)


def test_set_observation_switches_b(adj):
    """A problem pointed at a second observation buffer (set_observation)
    iterates exactly like one built on it; a layout mismatch is refused."""
    prob, wt, bl, db = _setup(adj, 96, 128, 3, "db2", "sym", 5, 1.0, 2e-3, 21)
    _, _, _, db2 = _setup(adj, 96, 128, 3, "db2", "sym", 5, 1.0, 2e-3, 22)
    f = adj.Fista(wt, bl, db2, 2e-3, 1.05)
    g = adj.Fista(wt, bl, db, 2e-3, 1.05)
    g.set_observation(db2)
    for _ in range(4):
        f.step()
        g.step()
    torch.cuda.synchronize()
    assert torch.equal(f.x, g.x) and torch.equal(f.y, g.y)
    with pytest.raises(ValueError):
        g.set_observation(torch.zeros(3, 3, device="cuda"))


def test_full_size_two_steps_sym(adj):
    """2048^2, CDF 9/7 J=5, symmetric BC, 15x15 sigma=3: two steps against the oracle."""
    rows = cols = 2048
    prob, wt, bl, db = _setup(adj, rows, cols, 5, "cdf97", "sym", 15, 3.0, 1e-3, 12)
    L = 1.01  # two steps at a fixed step size: parity does not need the estimated L_f
    f = adj.Fista(wt, bl, db, 1e-3, L)
    x, y, t = np.zeros(wt.logical_size), np.zeros(wt.logical_size), 1.0
    for k in range(2):
        x, y, t = ofista.fista_step(prob, x, y, t, L)
        f.step()
    assert rel_err(wt.unpack(f.x).cpu().numpy(), x) <= 1e-4
    assert rel_err(wt.unpack(f.y).cpu().numpy(), y) <= 1e-4


@pytest.mark.parametrize("w,mode,bc", [("cdf97", "sym", "sym"), ("db2", "per", "per")])
def test_pinv_gradient_variant(adj, w, mode, bc):
    """gradient="pinv" (W^dagger in place of W^*) follows the oracle's variant;
    it stalls above the exact-adjoint objective for a biorthogonal transform
    with symmetric boundaries and coincides with it for an orthogonal one with
    circular boundaries."""
    import dataclasses
    prob_e, wt, bl, db = _setup(adj, 96, 80, 2, w, mode, 7, 1.2, 2e-3, 31, bc=bc)
    prob_p = dataclasses.replace(prob_e, gradient="pinv")
    L = ofista.lipschitz(prob_e, random_vector(wt.logical_size, 2), iters=30)
    fe = adj.Fista(wt, bl, db, 2e-3, L)
    fp = adj.Fista(wt, bl, db, 2e-3, L, gradient="pinv")
    x, y, t = np.zeros(wt.logical_size), np.zeros(wt.logical_size), 1.0
    for k in range(1, 21):
        x, y, t = ofista.fista_step(prob_p, x, y, t, L)
        Fg = fp.step(objective=(k % 10 == 0))
        if k % 10 == 0:
            assert abs(Fg - prob_p.objective(x)) <= 1e-5 * prob_p.objective(x)
    assert rel_err(wt.unpack(fp.x).cpu().numpy(), x) <= 1e-4
    for _ in range(20):
        fe.step()
    for _ in range(130):
        fe.step()
        fp.step()
    Fe, Fp = fe.objective(), fp.objective()
    if mode == "sym":
        assert Fp > 1.1 * Fe
    else:
        assert abs(Fp - Fe) <= 1e-5 * Fe


def test_nonfinite_observation_is_reported(adj):
    """Fault injected on the host: a NaN in the observation b reaches the
    float64 objective through the residual, and the call returns
    ADJWT_ERR_NONFINITE instead of a number; the device status word stays
    clear and the context keeps computing."""
    rows = cols = 32
    wt = adj.WtPlan(rows, cols, 2, "db2", "per")
    taps = list(oblur.gaussian_psf(5, 1.0))
    bl = adj.BlurPlan(rows, cols, taps, taps, "per")
    b = wt.image(piecewise_smooth_image(rows, cols, 81))
    b[5, 7] = float("nan")
    f = adj.Fista(wt, bl, b, 1e-3, 1.0)
    with pytest.raises(adj.AdjwtError) as e:
        f.step(objective=True)
    assert e.value.code == -6
    with pytest.raises(adj.AdjwtError) as e:
        f.objective(torch.zeros_like(f.x))
    assert e.value.code == -6
    b[5, 7] = 0.5
    f.reset()
    assert np.isfinite(f.step(objective=True))
    assert adj.device_status() == 0


@pytest.mark.parametrize("rows,J,w,mode", [(256, 3, "db2", "sym"), (2048, 5, "cdf97", "sym"), (2048, 5, "cdf97", "per")])
def test_level_chain_fista_steps(adj, rows, J, w, mode):
    """FISTA with the prox epilogue in the level chain and without it: the
    iterates are bit-identical; the objective (whose |x| partials, float32
    within a tile, are summed in float64 over a different CTA split) agrees
    to float64 rounding."""
    prob, wt, bl, db = _setup(adj, rows, rows, J, w, mode, 9, 1.5, 1e-3, 3, bc="sym" if mode == "per" else None)
    res = []
    for chain in (True, False):
        wt.set_level_chain(chain)
        f = adj.Fista(wt, bl, db, 1e-3, 2.0)
        Fs = [f.step(objective=(k % 2 == 1)) for k in range(4)]
        torch.cuda.synchronize()
        res.append((f.x.clone(), f.y.clone(), [v for v in Fs if v is not None]))
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])
    for a, b in zip(res[0][2], res[1][2]):
        assert abs(a - b) <= 1e-13 * abs(b)
    assert adj.device_status() == 0
