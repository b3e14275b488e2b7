"""The batched FISTA engine: many problems of uneven sizes, depths, wavelets,
boundaries and PSF widths advanced in one persistent launch, checked against
the float64 oracle's FISTA (Eq. 1, the method cited in Sec. I-B) iteration by
iteration, and its bounded waits run out without faulting."""
import time

import numpy as np
import pytest
import torch

from oracle import blur as oblur
from oracle import fista as ofista
from synthetic_inputs import gaussian_noise, piecewise_smooth_image, random_taps, random_vector
from tests.gpu_util import image_dev, rel_err

pytestmark = pytest.mark.gpu

ADJWT_ERR_TIMEOUT = -8

# (rows, cols, levels, wavelet, wavelet boundary, PSF taps, sigma, blur boundary, gradient)
MIX = [
    (96, 96, 2, "db2", "sym", 5, 0.9, "sym", "adjoint"),
    (128, 112, 3, "db4", "zero", 9, 1.5, "zero", "adjoint"),
    (160, 160, 3, "cdf97", "sym", 15, 2.5, "sym", "adjoint"),
    (64, 64, 2, "haar", "per", 3, 0.8, "per", "adjoint"),
    (200, 136, 2, "cdf97", "zero", 11, 1.8, "sym", "pinv"),
    (128, 128, 4, "db2", "per", 7, 1.2, "per", "adjoint"),
    (90, 150, 3, "db4", "sym", 13, 2.0, "zero", "adjoint"),
    (120, 120, 3, "cdf97", "sym", 19, 3.0, "sym", "adjoint"),
    # non-palindromic taps under the symmetric boundary: the gathered-window
    # blur stage (the others take the TMA-window stage)
    (100, 84, 2, "db4", "sym", 7, None, "sym", "adjoint"),
]
LAM = 1e-3


@pytest.fixture(scope="module")
def adj():
    import paper_1707_02018_gb300 as adj
    adj.lib()
    return adj


def _problems(adj, mix=MIX, seed=900):
    out = []
    for i, (rows, cols, J, w, mode, k, sigma, bbc, grad) in enumerate(mix):
        p = oblur.gaussian_psf(k, sigma) if sigma is not None else random_taps(k, 77 + i)
        img = piecewise_smooth_image(rows, cols, seed + i)
        b = oblur.blur(img, p, p, bbc) + gaussian_noise((rows, cols), seed + 50 + i)
        prob = ofista.Problem(rows, cols, J, w, mode, p, p, bbc, b, LAM, gradient=grad)
        wt = adj.WtPlan(rows, cols, J, w, mode)
        bl = adj.BlurPlan(rows, cols, p, p, bbc)
        db = image_dev(wt, b)
        f = adj.Fista(wt, bl, db, LAM, 1.0, gradient=grad)
        L = 1.05 * f.lipschitz(wt.pack(random_vector(wt.logical_size, seed + 70 + i)), iters=30)
        f.set_lipschitz(L)
        out.append({"oracle": prob, "fista": f, "wt": wt, "bl": bl, "b": db, "L": L})
    return out


def test_batch_iterates_and_objectives_match_the_oracle(adj):
    """9 mixed problems, 6 iterations in one launch, then 4 more in a second:
    every iterate within 1e-4 (relative L2) of the float64 oracle after each
    launch, and the batched objective F(x_k) within 1e-5."""
    probs = _problems(adj)
    batch = adj.FistaBatch([p["fista"] for p in probs])
    info = batch.info()
    assert info["stages"] == sum(2 * m[2] + 2 for m in MIX)
    batch.reset()
    xs = [np.zeros(p["wt"].logical_size) for p in probs]
    ys = [x.copy() for x in xs]
    ts = [1.0] * len(probs)
    done = 0
    for iters in (6, 4):
        batch.run(iters)
        for i, p in enumerate(probs):
            for _ in range(iters):
                xs[i], ys[i], ts[i] = ofista.fista_step(p["oracle"], xs[i], ys[i], ts[i], p["L"])
        done += iters
        F = batch.objective().cpu().numpy()
        torch.cuda.synchronize()
        for i, p in enumerate(probs):
            xg = p["wt"].unpack(p["fista"].x).cpu().numpy()
            assert rel_err(xg, xs[i]) <= 1e-4, (i, done, rel_err(xg, xs[i]))
            Fo = p["oracle"].objective(xs[i])
            assert abs(F[i] - Fo) <= 1e-5 * Fo, (i, done, F[i], Fo)
    assert adj.device_status() == 0


# Stages of a few hundred tiles: W level 1 of 600 x 520 has 323 tiles, of
# 520 x 456 255; the blur stages 171 and 136 windows.
MIX_LARGE = [
    (600, 520, 3, "cdf97", "sym", 15, 2.0, "sym", "adjoint"),
    (520, 456, 2, "db2", "per", 7, 1.2, "per", "adjoint"),
    (96, 96, 2, "db4", "zero", 5, 0.9, "zero", "adjoint"),
]


def test_batch_of_large_stages_matches_the_oracle(adj):
    """Problems with stages of a few hundred tiles: every iterate within 1e-4
    of the float64 oracle after 5 iterations in one launch, and the
    objective within 1e-5."""
    probs = _problems(adj, MIX_LARGE, seed=1200)
    batch = adj.FistaBatch([p["fista"] for p in probs])
    batch.reset()
    batch.run(5)
    F = batch.objective().cpu().numpy()
    torch.cuda.synchronize()
    for i, p in enumerate(probs):
        x = np.zeros(p["wt"].logical_size)
        y, t = x.copy(), 1.0
        for _ in range(5):
            x, y, t = ofista.fista_step(p["oracle"], x, y, t, p["L"])
        xg = p["wt"].unpack(p["fista"].x).cpu().numpy()
        assert rel_err(xg, x) <= 1e-4, (i, rel_err(xg, x))
        Fo = p["oracle"].objective(x)
        assert abs(F[i] - Fo) <= 1e-5 * Fo, (i, F[i], Fo)
    assert adj.device_status() == 0


def test_batch_with_several_tiles_per_item_matches_one_problem_at_a_time(adj):
    """Eight 1048 x 984 problems: the W level-1 stage slot holds 8 x 1023
    tiles, over 16 per CTA of a full GPU, so the engine hands out its tiles
    two per item (the last item of each problem one).  After 8 iterations
    the engine's iterates equal fista_step's (one problem at a time, the
    per-level kernels) within float32 tolerance, and the batch needs fewer
    items per iteration than the eight problems batched one by one."""
    mix = [(1048, 984, 3, w, mode, 9, 1.5, mode, "adjoint")
           for w, mode in (("cdf97", "sym"), ("db2", "per"), ("db4", "sym"), ("cdf97", "zero"))] * 2
    probs = _problems(adj, mix, seed=1400)
    # alone, a problem's stages keep one tile per item
    single = sum(adj.FistaBatch([p["fista"]]).info()["items_per_iteration"] for p in probs)
    batch = adj.FistaBatch([p["fista"] for p in probs])
    assert batch.info()["items_per_iteration"] < single
    batch.reset()
    batch.run(8)
    torch.cuda.synchronize()
    got = [p["fista"].x.clone() for p in probs]
    for i, p in enumerate(probs):
        f = p["fista"]
        f.reset()
        for _ in range(8):
            f.step()
        torch.cuda.synchronize()
        r = float((got[i] - f.x).norm() / f.x.norm())
        assert r <= 1e-5, (i, r)
    assert adj.device_status() == 0


def test_batch_matches_one_problem_at_a_time(adj):
    """The engine and fista_step (one problem at a time, other kernels) give
    the same iterates within float32 tolerance after 10 iterations."""
    probs = _problems(adj)
    batch = adj.FistaBatch([p["fista"] for p in probs])
    batch.reset()
    batch.run(10)
    torch.cuda.synchronize()
    got = [p["fista"].x.clone() for p in probs]
    for i, p in enumerate(probs):
        f = p["fista"]
        f.reset()
        for _ in range(10):
            f.step()
        torch.cuda.synchronize()
        r = float((got[i] - f.x).norm() / f.x.norm())
        assert r <= 1e-5, (i, r)


def test_batch_wait_runs_out_and_the_launch_drains(adj):
    """A host-side setup in which the first stage waits for one that never
    runs: the bounded wait gives up after about a second, records
    ADJWT_ERR_TIMEOUT, every other CTA stops, and the context still computes
    (the next launch gives the oracle's iterates)."""
    probs = _problems(adj)[:3]
    batch = adj.FistaBatch([p["fista"] for p in probs])
    batch.reset()
    adj.device_status(clear=True)
    t0 = time.perf_counter()
    batch.wait_selftest()
    status = adj.device_status(clear=True)   # synchronises
    elapsed = time.perf_counter() - t0
    assert status == ADJWT_ERR_TIMEOUT
    assert 0.1 < elapsed < 60.0, elapsed
    assert adj.device_status() == 0
    batch.reset()
    batch.run(3)
    torch.cuda.synchronize()
    for i, p in enumerate(probs):
        x, y, t = np.zeros(p["wt"].logical_size), np.zeros(p["wt"].logical_size), 1.0
        for _ in range(3):
            x, y, t = ofista.fista_step(p["oracle"], x, y, t, p["L"])
        assert rel_err(p["wt"].unpack(p["fista"].x).cpu().numpy(), x) <= 1e-4
    assert adj.device_status() == 0


def test_batch_rejects_what_it_cannot_run(adj):
    p = oblur.gaussian_psf(5, 1.0)
    wt = adj.WtPlan(64, 64, 2, "db2", "ppd")
    bl = adj.BlurPlan(64, 64, p, p, "sym")
    f = adj.Fista(wt, bl, image_dev(wt, np.zeros((64, 64))), LAM, 1.0)
    with pytest.raises(adj.AdjwtError) as e:
        adj.FistaBatch([f])
    assert e.value.code == -2                 # SHAPE: redundant periodic reconstruction
    wide = oblur.gaussian_psf(27, 4.0)        # radius 13
    wt = adj.WtPlan(64, 64, 2, "db2", "sym")
    bl = adj.BlurPlan(64, 64, wide, wide, "sym")
    f = adj.Fista(wt, bl, image_dev(wt, np.zeros((64, 64))), LAM, 1.0)
    with pytest.raises(adj.AdjwtError) as e:
        adj.FistaBatch([f])
    assert e.value.code == -2


def test_rebuilt_batch_continues_the_runs(adj):
    """A batch rebuilt over a subset of the problems, with their x and y kept
    and the momentum set to where the first batch left it, continues the same
    FISTA sequences: the iterates after 6 + 4 iterations are bit-identical to
    10 iterations in one batch."""
    probs = _problems(adj)
    fs = [p["fista"] for p in probs]
    whole = adj.FistaBatch(fs)
    whole.reset()
    whole.run(10)
    torch.cuda.synchronize()
    want = [f.x.clone() for f in fs]
    whole.reset()
    whole.run(6)
    sub = [0, 2, 5, 7]
    keep = [fs[i] for i in sub]
    saved = [(f.x.clone(), f.y.clone()) for f in keep]
    part = adj.FistaBatch(keep)
    part.reset()
    for f, (x, y) in zip(keep, saved):
        f.x.copy_(x)
        f.y.copy_(y)
    part.set_momentum(6)
    part.run(4)
    torch.cuda.synchronize()
    for i, f in zip(sub, keep):
        assert torch.equal(f.x, want[i]), i
    assert adj.device_status() == 0
