"""Device-resident FISTA momentum (fista_step_device) and CUDA-graph replay.

The device path must reproduce the host-state iteration exactly (the same
t_k sequence, computed with correctly rounded float64 square roots on both
sides) and survive stream capture: a graph of several iterations over
several problems on their own streams, replayed, matches the oracle."""
import numpy as np
import pytest
import torch

from oracle import blur as oblur
from oracle import fista as ofista
from synthetic_inputs import gaussian_noise, piecewise_smooth_image
from tests.gpu_util import image_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def adj():
    import paper_1707_02018_gb300 as adj
    adj.lib()
    return adj


def _problem(adj, rows, cols, J, w, mode, k, sigma, lam, seed, L=None):
    bc = "per" if mode in ("per", "ppd") else mode
    p = oblur.gaussian_psf(k, sigma)
    img = piecewise_smooth_image(rows, cols, seed)
    b = oblur.blur(img, p, p, bc) + gaussian_noise((rows, cols), seed + 1)
    prob = ofista.Problem(rows, cols, J, w, mode, p, p, bc, b, lam)
    wt = adj.WtPlan(rows, cols, J, w, mode)
    bl = adj.BlurPlan(rows, cols, p, p, bc)
    db = image_dev(wt, b)
    f = adj.Fista(wt, bl, db, lam, L if L is not None else 1.0)
    return prob, wt, f


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_device_momentum_matches_host_state(adj):
    _, wt, f = _problem(adj, 160, 200, 3, "cdf97", "sym", 9, 1.5, 1e-3, 41, L=1.05)
    _, _, g = _problem(adj, 160, 200, 3, "cdf97", "sym", 9, 1.5, 1e-3, 41, L=1.05)
    f.reset()
    g.reset_device()
    obj = torch.zeros(1, dtype=torch.float64, device="cuda")
    for k in range(1, 16):
        Fh = f.step(objective=(k % 5 == 0))
        g.step_device(objective_out=obj if k % 5 == 0 else None)
        if k % 5 == 0:
            assert abs(float(obj) - Fh) <= 1e-12 * abs(Fh)
    torch.cuda.synchronize()
    assert torch.equal(f.x, g.x) and torch.equal(f.y, g.y)


@pytest.mark.parametrize("n_iters", [6])
def test_graph_of_iterations_over_problems(adj, n_iters):
    """Capture n_iters iterations of three problems (different sizes, wavelets
    and boundaries) on three streams, replay twice, compare with the oracle."""
    specs = [(96, 128, 3, "db2", "sym", 7, 1.0, 2e-3, 51), (128, 96, 2, "db4", "per", 9, 1.5, 1e-3, 52),
             (80, 72, 3, "cdf97", "zero", 5, 0.8, 3e-3, 53)]
    runs = []
    for sp in specs:
        prob, wt, f = _problem(adj, *sp)
        L = ofista.lipschitz(prob, np.random.default_rng(sp[-1]).standard_normal(wt.logical_size), iters=30)
        f.set_lipschitz(L)
        runs.append((prob, wt, f, L))
    streams = [torch.cuda.Stream() for _ in runs]
    objs = torch.zeros(len(runs), dtype=torch.float64, device="cuda")
    # warm-up outside capture (sets kernel attributes and occupancy caches)
    for (_, _, f, _), st in zip(runs, streams):
        f.reset_device(stream=st)
        f.step_device(stream=st)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    with torch.cuda.graph(graph, stream=cap):
        main = torch.cuda.current_stream()
        for st in streams:
            st.wait_stream(main)
        for i, ((_, _, f, _), st) in enumerate(zip(runs, streams)):
            for it in range(n_iters):
                f.step_device(objective_out=objs[i:i + 1] if it == n_iters - 1 else None, stream=st)
        for st in streams:
            main.wait_stream(st)
    for (_, _, f, _), st in zip(runs, streams):
        f.reset_device(stream=st)
    torch.cuda.synchronize()
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    for i, (prob, wt, f, L) in enumerate(runs):
        x, y, t = np.zeros(wt.logical_size), np.zeros(wt.logical_size), 1.0
        for _ in range(2 * n_iters):
            x, y, t = ofista.fista_step(prob, x, y, t, L)
        assert rel_err(wt.unpack(f.x).cpu().numpy(), x) <= 1e-4
        assert abs(float(objs[i]) - prob.objective(x)) <= 1e-5 * prob.objective(x)
    assert adj.device_status() == 0
