"""Differentiation through the solve of Eq. 1 on the GPU against the float64
oracle: dR/dsigma, the elementwise backward kernels, and the unrolled-FISTA
gradients with respect to lambda, sigma and b (oracle: its reverse mode,
itself pinned by central differences in tests/test_oracle_unrolled.py)."""
import numpy as np
import pytest
import torch

from oracle import blur as oblur
from oracle import fista as ofista
from oracle import unrolled as ounr
from oracle.filters import filter_bank
from oracle.layout import num_coeffs
from synthetic_inputs import gaussian_noise, piecewise_smooth_image, random_vector
from tests.gpu_util import assert_close, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def adj():
    import paper_1707_02018_gb300 as adj
    adj.lib()
    return adj


@pytest.mark.parametrize("bc", ["zero", "sym", "per"])
def test_dR_dsigma_matches_oracle(adj, bc):
    rows, cols, k, sigma = 64, 72, 9, 1.6
    u = random_vector((rows, cols), 5)
    g, dg = adj.gaussian_taps(k, sigma)
    p1 = adj.BlurPlan(rows, cols, dg, g, bc)
    p2 = adj.BlurPlan(rows, cols, g, dg, bc)
    ud = p1.image(u)
    got = adj.axpby(1.0, adj.blur(p1, ud), 1.0, adj.blur(p2, ud))[:, :cols].double().cpu().numpy()
    S = ounr.Setup(rows, cols, 1, "db2", "sym", k, sigma, bc, np.zeros((rows, cols)), 0.0, 1.0)
    assert_close(got, S.dR(u), what=f"dR/dsigma {bc}")


def test_elementwise_backward_kernels(adj):
    n = 100003
    x = torch.randn(n, device="cuda")
    x[::3] = 0.0
    g = torch.randn(n, device="cuda")
    zbar, s = adj.prox_vjp(x, g)
    xn, gn = x.cpu().numpy(), g.cpu().numpy()
    assert np.array_equal(zbar.cpu().numpy(), np.where(xn != 0, gn, 0.0).astype(np.float32))
    assert abs(float(s) - float(np.sum(np.sign(xn).astype(np.float64) * gn))) <= 1e-12 * np.sum(np.abs(gn))
    out = adj.axpby(0.5, x, -2.0, g)
    assert np.allclose(out.cpu().numpy(), 0.5 * xn - 2.0 * gn, rtol=1e-6, atol=1e-6)
    d = adj.dot(x, g)
    assert abs(float(d) - float(np.dot(xn.astype(np.float64), gn))) <= 1e-12 * float(np.abs(xn) @ np.abs(gn))
    # pitched: only the first cols of each row count
    img = torch.randn(7, 12, device="cuda")
    d2 = adj.dot(img, img, rows=7, cols=9, pitch=12)
    ref = float(np.sum(img.cpu().numpy()[:, :9].astype(np.float64) ** 2))
    assert abs(float(d2) - ref) <= 1e-12 * ref
    assert adj.device_status() == 0


def _problem(adj, rows, cols, levels, wavelet, mode, bc, k, sigma, lam, seed):
    img = piecewise_smooth_image(rows, cols, seed)
    q = oblur.gaussian_psf(k, sigma)
    b = oblur.blur(img, q, q, bc) + gaussian_noise((rows, cols), seed + 1, 1e-2)
    nco = num_coeffs(rows, cols, levels, filter_bank(wavelet).L, mode)
    prob = ofista.Problem(rows, cols, levels, wavelet, mode, q, q, bc, b, lam)
    L = ofista.lipschitz(prob, np.random.default_rng(seed).standard_normal(nco), iters=40)
    S = ounr.Setup(rows, cols, levels, wavelet, mode, k, sigma, bc, b, lam, L)
    return S, img, nco


@pytest.mark.parametrize("wavelet,mode,bc", [("cdf97", "sym", "sym"), ("db2", "per", "per")])
def test_unrolled_gradients_match_oracle(adj, wavelet, mode, bc):
    from paper_1707_02018_gb300.unrolled import UnrolledFista
    rows = cols = 64
    levels, k, sigma, lam, steps = 3, 5, 1.2, 0.02, 10
    S, img, nco = _problem(adj, rows, cols, levels, wavelet, mode, bc, k, sigma, lam, 31)
    want = ounr.unrolled_grads(S, steps, img, nco)
    wt = adj.WtPlan(rows, cols, levels, wavelet, mode)
    bdev = wt.image(S.b)
    un = UnrolledFista(rows, cols, levels, wavelet, mode, k, sigma, bc, bdev, lam, S.L)
    got = un.grads(steps, wt.image(img), checkpoint_every=3)
    loss, dlam, dsig, db = got
    db_np = db[:, :cols].double().cpu().numpy()
    print(f"\n{wavelet}/{mode}: loss {loss:.6e} vs {want[0]:.6e}; dlam {dlam:.6e} vs {want[1]:.6e}; "
          f"dsigma {dsig:.6e} vs {want[2]:.6e}; db rel L2 {rel_err(db_np, want[3]):.3e}")
    # float32 iterates against float64: observed 5e-7 (loss, dlam), 1e-7
    # (dsigma) and 1.5e-6 (dl/db, relative L2); the bounds leave ~7x
    assert abs(loss - want[0]) <= 1e-5 * abs(want[0])
    assert abs(dlam - want[1]) <= 1e-5 * abs(want[1])
    assert abs(dsig - want[2]) <= 1e-5 * abs(want[2])
    assert rel_err(db_np, want[3]) <= 1e-5
    # checkpointing recomputes the same iterates: bit-identical results
    again = un.grads(steps, wt.image(img), checkpoint_every=1)
    once = un.grads(steps, wt.image(img), checkpoint_every=steps)
    for other in (again, once):
        assert other[0] == loss and other[1] == dlam and other[2] == dsig and torch.equal(other[3], db)
    # the one-call backward step (fista_vjp_step) against the same step built
    # from the separate library calls: the same kernels, so the same values up
    # to the order of the float64 accumulation of dl/dtau and dl/dsigma
    lp, dlp, dsp, dbp = un.grads(steps, wt.image(img), checkpoint_every=3, fused=False)
    assert lp == loss
    assert abs(dlp - dlam) <= 1e-9 * abs(dlam) and abs(dsp - dsig) <= 1e-9 * abs(dsig)
    assert rel_err(dbp[:, :cols].double().cpu().numpy(), db_np) <= 1e-6
    assert adj.device_status() == 0


def test_autograd_node(adj):
    from paper_1707_02018_gb300.unrolled import UnrolledFista, unrolled_loss
    rows = cols = 48
    levels, k, sigma, lam, steps = 2, 5, 1.0, 0.03, 6
    S, img, nco = _problem(adj, rows, cols, levels, "db2", "sym", "sym", k, sigma, lam, 41)
    wt = adj.WtPlan(rows, cols, levels, "db2", "sym")
    bdev = wt.image(S.b).requires_grad_(True)
    lam_t = torch.tensor(lam, dtype=torch.float64, requires_grad=True)
    sig_t = torch.tensor(sigma, dtype=torch.float64, requires_grad=True)
    spec = (rows, cols, levels, "db2", "sym", k, "sym")
    loss = unrolled_loss(lam_t, sig_t, bdev, wt.image(img), spec, steps, S.L)
    (2.0 * loss).backward()
    un = UnrolledFista(rows, cols, levels, "db2", "sym", k, sigma, "sym", wt.image(S.b), lam, S.L)
    l2, dl, ds, db = un.grads(steps, wt.image(img))
    assert float(loss.detach()) == l2
    assert float(lam_t.grad) == 2.0 * dl and float(sig_t.grad) == 2.0 * ds
    assert torch.equal(bdev.grad, adj.axpby(2.0, db, 0.0, db))


@pytest.mark.parametrize("steps,every,bc,mode", [(1, None, "zero", "zero"), (4, 9, "sym", "sym"), (5, 2, "per", "per")])
def test_unrolled_edge_cases(adj, steps, every, bc, mode):
    """One iteration, checkpoints sparser than the iterations, and the ZERO
    and PER blur boundaries, against the oracle's reverse mode."""
    from paper_1707_02018_gb300.unrolled import UnrolledFista
    rows = cols = 32
    S, img, nco = _problem(adj, rows, cols, 2, "db2", mode, bc, 5, 1.1, 0.02, 61 + steps)
    want = ounr.unrolled_grads(S, steps, img, nco)
    wt = adj.WtPlan(rows, cols, 2, "db2", mode)
    un = UnrolledFista(rows, cols, 2, "db2", mode, 5, 1.1, bc, wt.image(S.b), 0.02, S.L)
    loss, dlam, dsig, db = un.grads(steps, wt.image(img), checkpoint_every=every)
    assert abs(loss - want[0]) <= 1e-5 * abs(want[0])
    assert abs(dlam - want[1]) <= 1e-5 * max(abs(want[1]), 1e-6)
    assert abs(dsig - want[2]) <= 1e-5 * max(abs(want[2]), 1e-6)
    assert rel_err(db[:, :cols].double().cpu().numpy(), want[3]) <= 1e-5


def test_vjp_step_argument_errors(adj):
    """fista_vjp_step rejects, before any launch, a derivative plan of another
    image, dsigma without the plans, a small workspace and the W^dagger
    iteration (its backward would not be the chain rule's A^*)."""
    rows = cols = 32
    S, img, nco = _problem(adj, rows, cols, 2, "db2", "sym", "sym", 5, 1.1, 0.02, 71)
    wt = adj.WtPlan(rows, cols, 2, "db2", "sym")
    g, dg = adj.gaussian_taps(5, 1.1)
    R = adj.BlurPlan(rows, cols, g, g, "sym")
    dR = (adj.BlurPlan(rows, cols, dg, g, "sym"), adj.BlurPlan(rows, cols, g, dg, "sym"))
    other = (adj.BlurPlan(rows, 16, dg, g, "sym"), adj.BlurPlan(rows, 16, g, dg, "sym"))
    b = wt.image(S.b)
    f = adj.Fista(wt, R, b, 0.02, S.L)
    ws = f.vjp_workspace()
    v = [torch.zeros(wt.num_coeffs, device="cuda") for _ in range(4)]
    acc = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(adj.AdjwtError) as e:
        adj.fista_vjp_step(f, other, v[0], v[1], 0.5, v[2], v[3], None, acc[0:1], acc[1:2], ws)
    assert e.value.code == -2
    with pytest.raises(adj.AdjwtError) as e:
        adj.fista_vjp_step(f, None, v[0], v[1], 0.5, v[2], v[3], None, acc[0:1], acc[1:2], ws)
    assert e.value.code == -1
    with pytest.raises(adj.AdjwtError) as e:
        adj.fista_vjp_step(f, dR, v[0], v[1], 0.5, v[2], v[3], None, acc[0:1], acc[1:2], ws[:-256])
    assert e.value.code == -7
    fp = adj.Fista(wt, R, b, 0.02, S.L, gradient="pinv")
    with pytest.raises(adj.AdjwtError) as e:
        adj.fista_vjp_step(fp, dR, v[0], v[1], 0.5, v[2], v[3], None, acc[0:1], acc[1:2], fp.vjp_workspace())
    assert e.value.code == -1
    # the valid call goes through and leaves finite accumulators
    adj.fista_vjp_step(f, dR, v[0], v[1], 0.5, v[2], v[3], None, acc[0:1], acc[1:2], ws)
    assert torch.isfinite(acc).all()
