"""Parity of the CUDA W, W^* and W^dagger with the float64 oracle (Sec. I-A, Eq. 2-4)."""
import numpy as np
import pytest
import torch

from oracle import wavelet as owt
from synthetic_inputs import piecewise_smooth_image, random_vector
from tests.gpu_util import assert_close, image_dev, to_host_image

pytestmark = pytest.mark.gpu

WAVELETS = ["haar", "db2", "db4", "cdf97"]
MODES = ["zero", "sym", "ppd", "per"]
# several tiles with ragged tails, thin images, tiny images (N <= 2L': gather path)
SHAPES = [(64, 48, 2), (70, 45, 3), (33, 97, 2), (5, 7, 2), (1, 1, 1), (2, 3, 1), (19, 130, 1)]


@pytest.fixture(scope="module")
def adj():
    import paper_1707_02018_gb300 as adj
    adj.lib()
    return adj


def _shapes(mode):
    out = []
    for r, c, J in SHAPES:
        if mode == "per":
            r, c = r + (-r) % 2 ** J, c + (-c) % 2 ** J
        out.append((r, c, J))
    return out


@pytest.mark.parametrize("w", WAVELETS)
@pytest.mark.parametrize("mode", MODES)
def test_adjoint_analysis_synthesis_parity(adj, w, mode):
    for rows, cols, J in _shapes(mode):
        plan = adj.WtPlan(rows, cols, J, w, mode)
        img = random_vector((rows, cols), rows * 1000 + cols)
        dimg = image_dev(plan, img)
        got = adj.wt_synth_adjoint(plan, dimg)
        torch.cuda.synchronize()
        want = owt.wt_adjoint(img, J, w, mode)
        assert_close(plan.unpack(got).cpu().numpy(), want, what=f"W^* {w} {mode} {rows}x{cols} J{J}")
        # padding of every band is written as zero
        assert float((got.abs().sum() - plan.unpack(got).abs().sum()).abs()) < 1e-3 * float(got.abs().sum() + 1)
        got = adj.wt_analysis(plan, dimg)
        want = owt.wt_pinv(img, J, w, mode)
        assert_close(plan.unpack(got).cpu().numpy(), want, what=f"W^dagger {w} {mode} {rows}x{cols}")
        x = random_vector(plan.logical_size, rows + cols)
        out = adj.wt_synth(plan, plan.pack(x))
        want = owt.wt_synth(x, rows, cols, J, w, mode)
        assert_close(to_host_image(out, rows, cols), want, what=f"W {w} {mode} {rows}x{cols}")


@pytest.mark.parametrize("w", WAVELETS)
@pytest.mark.parametrize("mode", MODES)
def test_large_levels_interior_and_border_kernels(adj, w, mode):
    """Persistent TMA kernels: on levels they cover whole (512 x 1024 under
    PER / ZERO) and, on levels of at least 1024 x 1024, on the tiles they can
    take with the tiled kernel on the rest (levels of at least 1536 x 1536)."""
    for rows, cols, J in [(1600, 1664, 2), (512, 1024, 3)]:
        plan = adj.WtPlan(rows, cols, J, w, mode)
        x = random_vector(plan.logical_size, rows * 7 + cols)
        out = adj.wt_synth(plan, plan.pack(x))
        want = owt.wt_synth(x, rows, cols, J, w, mode)
        assert_close(to_host_image(out, rows, cols), want, what=f"W {w} {mode} {rows}x{cols} J{J}")
        img = random_vector((rows, cols), rows + 3 * cols)
        got = adj.wt_synth_adjoint(plan, image_dev(plan, img))
        assert_close(plan.unpack(got).cpu().numpy(), owt.wt_adjoint(img, J, w, mode),
                     what=f"W^* {w} {mode} {rows}x{cols} J{J}")
        got = adj.wt_analysis(plan, image_dev(plan, img))
        assert_close(plan.unpack(got).cpu().numpy(), owt.wt_pinv(img, J, w, mode),
                     what=f"W^dagger {w} {mode} {rows}x{cols} J{J}")
    assert adj.device_status() == 0


@pytest.mark.parametrize("w,mode", [("cdf97", "sym"), ("db2", "per"), ("db4", "zero"), ("cdf97", "ppd")])
def test_large_levels_tiled_only(adj, w, mode):
    """Every level forced onto the tiled kernels (the TMA kernels switched off
    for W and for W^* / W^dagger) on levels the size rule would give to the
    TMA kernels: same operators within the float32 tolerance."""
    rows, cols, J = 1600, 1664, 2
    plan = adj.WtPlan(rows, cols, J, w, mode)
    assert plan.tma_levels()["synth"][0] and plan.tma_levels()["analysis"][0]
    for j in range(1, J + 1):
        for op in ("synth", "analysis", "prox"):
            plan.set_tma(op, j, False)
    assert not any(any(v) for v in plan.tma_levels().values())
    x = random_vector(plan.logical_size, 17)
    out = adj.wt_synth(plan, plan.pack(x))
    assert_close(to_host_image(out, rows, cols), owt.wt_synth(x, rows, cols, J, w, mode), what=f"W tiled {w} {mode}")
    img = random_vector((rows, cols), 19)
    got = adj.wt_synth_adjoint(plan, image_dev(plan, img))
    assert_close(plan.unpack(got).cpu().numpy(), owt.wt_adjoint(img, J, w, mode), what=f"W^* tiled {w} {mode}")
    got = adj.wt_analysis(plan, image_dev(plan, img))
    assert_close(plan.unpack(got).cpu().numpy(), owt.wt_pinv(img, J, w, mode), what=f"W^dagger tiled {w} {mode}")
    assert adj.device_status() == 0


def test_autotune_and_its_cache(adj):
    """Autotuning measures every eligible level, leaves the operators exact,
    and a later plan of the same size class starts from the stored choice."""
    rows, cols, J, w, mode = 1600, 1664, 3, "cdf97", "sym"
    plan = adj.WtPlan(rows, cols, J, w, mode)
    assert plan.autotune(reps=3) is False
    chosen = plan.tma_levels()
    x = random_vector(plan.logical_size, 23)
    out = adj.wt_synth(plan, plan.pack(x))
    assert_close(to_host_image(out, rows, cols), owt.wt_synth(x, rows, cols, J, w, mode), what="W after autotune")
    img = random_vector((rows, cols), 29)
    got = adj.wt_synth_adjoint(plan, image_dev(plan, img))
    assert_close(plan.unpack(got).cpu().numpy(), owt.wt_adjoint(img, J, w, mode), what="W^* after autotune")
    caps = plan.tma_ctas()
    again = adj.WtPlan(rows, cols, J, w, mode)
    assert again.tma_levels() == chosen        # applied at creation
    assert again.tma_ctas() == caps
    assert again.autotune(reps=3) is True      # and not measured again
    assert again.tma_levels() == chosen
    print("\nautotune 1600x1664 J3 cdf97 sym:", chosen, caps)


@pytest.mark.parametrize("mode", ["sym", "per"])
@pytest.mark.parametrize("ctas", [1, 2])
def test_tma_cta_cap_gives_the_same_operators(adj, mode, ctas):
    """The TMA kernels capped at 1 or 2 resident CTAs per SM (every CTA then
    walks more tiles through its copy pipeline) give bit-identical W, W^* and
    FISTA iterates with the prox epilogue (each tile's arithmetic does not
    depend on which CTA runs it; the default path is held to the oracle by
    the tests above)."""
    from oracle import blur as oblur
    rows, cols, J, w = 2048, 2048, 3, "cdf97"
    plan = adj.WtPlan(rows, cols, J, w, mode)
    assert plan.tma_levels()["synth"][0] and plan.tma_levels()["prox"][0]
    x = plan.pack(random_vector(plan.logical_size, 31))
    img = image_dev(plan, random_vector((rows, cols), 37))
    p = oblur.gaussian_psf(9, 1.5)
    bl = adj.BlurPlan(rows, cols, p, p, mode)
    b = image_dev(plan, piecewise_smooth_image(rows, cols, 41))

    def run():
        f = adj.Fista(plan, bl, b, 1e-3, 1.0)
        f.step()
        f.step()
        return adj.wt_synth(plan, x).clone(), adj.wt_synth_adjoint(plan, img).clone(), f.x.clone()

    want = run()
    for op in ("synth", "analysis", "prox"):
        plan.set_tma_ctas(op, 1, ctas)
    assert plan.tma_ctas()["prox"][0] == ctas
    got = run()
    for g_, w_, what in zip(got, want, ("W", "W^*", "FISTA x_2")):
        assert torch.equal(g_, w_), what
    assert adj.device_status() == 0


@pytest.mark.parametrize("mode", ["sym", "per", "zero"])
def test_full_size_cdf97_five_levels(adj, mode):
    """The 2048 x 2048, 5-level CDF 9/7 operators of the bench, compared in full."""
    rows = cols = 2048
    plan = adj.WtPlan(rows, cols, 5, "cdf97", mode)
    img = piecewise_smooth_image(rows, cols, 11)
    got = adj.wt_synth_adjoint(plan, image_dev(plan, img))
    want = owt.wt_adjoint(img, 5, "cdf97", mode)
    assert_close(plan.unpack(got).cpu().numpy(), want, what=f"W^* 2048 {mode}")
    x = random_vector(plan.logical_size, 5)
    out = adj.wt_synth(plan, plan.pack(x))
    want = owt.wt_synth(x, rows, cols, 5, "cdf97", mode)
    assert_close(to_host_image(out, rows, cols), want, what=f"W 2048 {mode}")


@pytest.mark.parametrize("w", WAVELETS)
@pytest.mark.parametrize("mode", MODES)
def test_gpu_dot_product_and_reconstruction(adj, w, mode):
    rows, cols, J = (96, 64, 3)
    plan = adj.WtPlan(rows, cols, J, w, mode)
    x = plan.pack(random_vector(plan.logical_size, 1))
    yimg = image_dev(plan, random_vector((rows, cols), 2))
    Wx = adj.wt_synth(plan, x)
    Wty = adj.wt_synth_adjoint(plan, yimg)
    lhs = float((Wx[:, :cols].double() * yimg[:, :cols].double()).sum())
    rhs = float((x.double() * Wty.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    u = image_dev(plan, piecewise_smooth_image(rows, cols, 3))
    rec = adj.wt_synth(plan, adj.wt_analysis(plan, u))
    assert float((rec - u)[:, :cols].abs().max()) < 1e-5


def test_repeated_calls_and_streams(adj):
    """Plans are reusable and stream-ordered: two streams, same plan, same result."""
    plan = adj.WtPlan(130, 70, 3, "db4", "sym")
    img = image_dev(plan, random_vector((130, 70), 9))
    ref = adj.wt_synth_adjoint(plan, img).clone()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s1):
        a = adj.wt_synth_adjoint(plan, img)
    with torch.cuda.stream(s2):
        b = adj.wt_synth_adjoint(plan, img)
    torch.cuda.synchronize()
    assert torch.equal(a, ref) and torch.equal(b, ref)


def test_errors_reach_python(adj):
    plan = adj.WtPlan(16, 16, 1, "db2", "sym")
    buf = torch.zeros(4096, dtype=torch.float32, device="cuda")
    img = buf[:256].view(16, 16)
    with pytest.raises(adj.AdjwtError) as e:
        adj.wt_synth_adjoint(plan, img, coeffs=buf[64:64 + plan.num_coeffs])   # output aliases input
    assert e.value.code == -4
    with pytest.raises(adj.AdjwtError):
        adj.WtPlan(12, 16, 3, "db2", "per")


@pytest.mark.parametrize("rows,cols,J,w,mode", [
    (2048, 2048, 5, "cdf97", "sym"), (2048, 2048, 5, "cdf97", "per"), (2048, 2048, 5, "cdf97", "zero"),
    (256, 256, 3, "db2", "sym"), (300, 211, 4, "db4", "zero"), (70, 45, 3, "haar", "per"),
    (64, 48, 2, "cdf97", "ppd"), (5, 7, 2, "db2", "sym")])
def test_level_chain_equals_per_level_launches(adj, rows, cols, J, w, mode):
    """With the level chain switched on, the deep levels run as one launch.  The
    chain runs the same tile code as the per-level launches, so W, W^* and
    W^dagger are bit-identical with the chain on and off, and still match
    the oracle."""
    if mode == "per":
        rows, cols = rows + (-rows) % 2 ** J, cols + (-cols) % 2 ** J
    plan = adj.WtPlan(rows, cols, J, w, mode)
    assert plan.chain_start() == {"synth": 0, "analysis": 0, "prox": 0}   # off by default
    plan.set_level_chain(True)
    starts = plan.chain_start()
    x = plan.pack(random_vector(plan.logical_size, rows + 5 * cols))
    img = image_dev(plan, random_vector((rows, cols), 3 * rows + cols))
    on = [adj.wt_synth(plan, x).clone(), adj.wt_synth_adjoint(plan, img).clone(), adj.wt_analysis(plan, img).clone()]
    plan.set_level_chain(False)
    assert plan.chain_start() == {"synth": 0, "analysis": 0, "prox": 0}
    off = [adj.wt_synth(plan, x), adj.wt_synth_adjoint(plan, img), adj.wt_analysis(plan, img)]
    torch.cuda.synchronize()
    for name, a, b in zip(("W", "W^*", "W^dagger"), on, off):
        assert torch.equal(a, b), f"{name} {rows}x{cols} J{J} {w} {mode}: chain differs from per-level launches"
    if rows * cols <= 300 * 300:
        assert_close(plan.unpack(on[1]).cpu().numpy(), owt.wt_adjoint(img[:, :cols].double().cpu().numpy(), J, w, mode),
                     what=f"W^* chain {w} {mode}")
    assert adj.device_status() == 0
    print(f"\nchain start {rows}x{cols} J{J} {w} {mode}: {starts}")


def test_level_chain_is_where_the_rule_puts_it(adj):
    """2048^2, 5 levels: levels 2..5 chained under SYM and ZERO (level 1 runs
    on the TMA kernels); PER hands levels 1-3 to the TMA kernels and chains
    4..5 of W (W^* runs level 1 alone on them, so it chains 2..5); PPD
    reconstruction has no chain; small images chain every level."""
    def starts(*args):
        plan = adj.WtPlan(*args)
        plan.set_level_chain(True)
        return plan.chain_start()
    for mode, want in (("sym", (2, 2)), ("zero", (2, 2)), ("per", (4, 2))):
        s = starts(2048, 2048, 5, "cdf97", mode)
        assert s == {"synth": want[0], "analysis": want[1], "prox": want[1]}, (mode, s)
    assert starts(512, 512, 4, "cdf97", "ppd")["synth"] == 0
    assert starts(256, 256, 3, "db2", "sym") == {"synth": 1, "analysis": 1, "prox": 1}
    assert starts(256, 256, 1, "db2", "sym") == {"synth": 0, "analysis": 0, "prox": 0}
