"""Child process of tests/test_gpu_bounds_checked.py: runs the operators of the
library build named by ADJWT_LIBRARY (the bounds-checked one) on parity cases
and prints one JSON line: the relative errors against the float64 oracle and
the device status word after each group."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import paper_1707_02018_gb300 as adj  # noqa: E402
from oracle import blur as oblur  # noqa: E402
from oracle import fista as ofista  # noqa: E402
from oracle import wavelet as owt  # noqa: E402
from synthetic_inputs import gaussian_noise, piecewise_smooth_image, random_vector  # noqa: E402
from tests.gpu_util import image_dev, rel_err, to_host_image  # noqa: E402


def main():
    assert os.environ.get("ADJWT_LIBRARY"), "run with ADJWT_LIBRARY set"
    adj.lib()
    assert adj._lib.LIB_PATH == os.environ["ADJWT_LIBRARY"]
    out = {"errors": {}, "status": {}}
    adj.device_status(clear=True)
    cases = [(70, 45, 3, "db4", "sym"), (64, 48, 2, "cdf97", "zero"), (5, 7, 2, "db2", "sym"),
             (96, 64, 3, "haar", "per"), (33, 97, 2, "db2", "ppd"), (1600, 1664, 2, "cdf97", "sym"),
             (2048, 2048, 5, "cdf97", "per")]
    for rows, cols, J, w, mode in cases:
        plan = adj.WtPlan(rows, cols, J, w, mode)
        img = random_vector((rows, cols), rows + cols)
        got = plan.unpack(adj.wt_synth_adjoint(plan, image_dev(plan, img))).cpu().numpy()
        out["errors"][f"W* {rows}x{cols} {w} {mode}"] = rel_err(got, owt.wt_adjoint(img, J, w, mode))
        x = random_vector(plan.logical_size, rows * cols)
        got = to_host_image(adj.wt_synth(plan, plan.pack(x)), rows, cols)
        out["errors"][f"W {rows}x{cols} {w} {mode}"] = rel_err(got, owt.wt_synth(x, rows, cols, J, w, mode))
    torch.cuda.synchronize()
    out["status"]["wavelet"] = adj.device_status(clear=True)
    for rows, cols, k, bc in [(200, 300, 15, "sym"), (37, 53, 9, "per"), (2048, 2048, 15, "zero")]:
        p = oblur.gaussian_psf(k, 2.0)
        plan = adj.BlurPlan(rows, cols, p, p, bc)
        u = random_vector((rows, cols), 7)
        b = random_vector((rows, cols), 8)
        g = adj.blur_normal(plan, plan.image(u), plan.image(b))
        got = g[0] if isinstance(g, tuple) else g
        want = oblur.blur_adjoint(oblur.blur(u, p, p, bc) - b, p, p, bc)
        out["errors"][f"R*(Ru-b) {rows}x{cols} {bc}"] = rel_err(got[:, :cols].double().cpu().numpy(), want)
        fused = adj.blur_normal(plan, plan.image(u), plan.image(b), scratch=False)   # the fused tiled kernel
        fused = fused[0] if isinstance(fused, tuple) else fused
        out["errors"][f"R*(Ru-b) fused {rows}x{cols} {bc}"] = rel_err(fused[:, :cols].double().cpu().numpy(), want)
    torch.cuda.synchronize()
    out["status"]["blur"] = adj.device_status(clear=True)
    # FISTA (level-1 TMA W* + prox at 2048^2) and the batched engine
    rows = cols = 2048
    p = oblur.gaussian_psf(15, 3.0)
    img = piecewise_smooth_image(rows, cols, 5)
    b = oblur.blur(img, p, p, "sym") + gaussian_noise((rows, cols), 6)
    wt = adj.WtPlan(rows, cols, 5, "cdf97", "sym")
    bl = adj.BlurPlan(rows, cols, p, p, "sym")
    f = adj.Fista(wt, bl, image_dev(wt, b), 1e-3, 2.0)
    for _ in range(2):
        f.step()
    prob = ofista.Problem(rows, cols, 5, "cdf97", "sym", p, p, "sym", b, 1e-3)
    x, y, t = np.zeros(wt.logical_size), np.zeros(wt.logical_size), 1.0
    for _ in range(2):
        x, y, t = ofista.fista_step(prob, x, y, t, 2.0)
    out["errors"]["FISTA 2048 sym, 2 steps"] = rel_err(wt.unpack(f.x).cpu().numpy(), x)
    small = []
    for i, (n, J, wv, k) in enumerate([(96, 3, "db4", 7), (130, 2, "cdf97", 11), (64, 3, "db2", 5)]):
        pp = oblur.gaussian_psf(k, 1.5)
        wti = adj.WtPlan(n, n, J, wv, "sym")
        bli = adj.BlurPlan(n, n, pp, pp, "sym")
        bi = oblur.blur(piecewise_smooth_image(n, n, 30 + i), pp, pp, "sym")
        small.append((adj.Fista(wti, bli, image_dev(wti, bi), 1e-3, 2.0),
                      ofista.Problem(n, n, J, wv, "sym", pp, pp, "sym", bi, 1e-3), wti))
    batch = adj.FistaBatch([s[0] for s in small])
    batch.reset()
    batch.run(3)
    torch.cuda.synchronize()
    for fi, pr, wti in small:
        xo, yo, to = np.zeros(wti.logical_size), np.zeros(wti.logical_size), 1.0
        for _ in range(3):
            xo, yo, to = ofista.fista_step(pr, xo, yo, to, 2.0)
        out["errors"][f"batch {wti.rows}"] = rel_err(wti.unpack(fi.x).cpu().numpy(), xo)
    torch.cuda.synchronize()
    out["status"]["fista"] = adj.device_status(clear=True)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
