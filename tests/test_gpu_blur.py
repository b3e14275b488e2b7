"""Parity of the CUDA R, R^* and fused R^*(R u - b) with the float64 oracle."""
import numpy as np
import pytest
import torch

from oracle import blur as oblur
from synthetic_inputs import piecewise_smooth_image, random_taps, random_vector
from tests.gpu_util import assert_close, image_dev, to_host_image

pytestmark = pytest.mark.gpu

BCS = ["zero", "sym", "per"]
SHAPES = [(64, 48), (70, 45), (33, 100), (5, 3), (1, 1), (2, 7)]
PSFS = [("asym5x3", 5, 3), ("gauss9", 9, 9), ("asym15x7", 15, 7)]


@pytest.fixture(scope="module")
def adj():
    import paper_1707_02018_gb300 as adj
    adj.lib()
    return adj


def _taps(name, kr, kc):
    if name.startswith("gauss"):
        p = oblur.gaussian_psf(kr, 1.5)
        return p, p
    return random_taps(kr, kr * 7 + 1), random_taps(kc, kc * 5 + 2)


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("psf", PSFS, ids=[p[0] for p in PSFS])
def test_blur_family_parity(adj, bc, psf):
    pr, pc = _taps(*psf)
    for rows, cols in SHAPES:
        plan = adj.BlurPlan(rows, cols, pr, pc, bc)
        u = random_vector((rows, cols), rows * 31 + cols)
        b = random_vector((rows, cols), rows * 37 + cols)
        du, db = image_dev(plan, u), image_dev(plan, b)
        what = f"{bc} {psf[0]} {rows}x{cols}"
        assert_close(to_host_image(adj.blur(plan, du), rows, cols), oblur.blur(u, pr, pc, bc), what="R " + what)
        assert_close(to_host_image(adj.blur_adjoint(plan, du), rows, cols), oblur.blur_adjoint(u, pr, pc, bc),
                     what="R^* " + what)
        g, half = adj.blur_normal(plan, du, db, want_norm=True)
        gw, hw = oblur.blur_normal(u, b, pr, pc, bc)
        assert_close(to_host_image(g, rows, cols), gw, what="R^*(Ru-b) " + what)
        assert abs(float(half) - hw) <= 1e-5 * hw


@pytest.mark.parametrize("bc", BCS)
def test_full_size_15x15(adj, bc):
    rows = cols = 2048
    p = oblur.gaussian_psf(15, 3.0)
    plan = adj.BlurPlan(rows, cols, p, p, bc)
    u = piecewise_smooth_image(rows, cols, 21)
    b = piecewise_smooth_image(rows, cols, 22)
    du = image_dev(plan, u)
    g, half = adj.blur_normal(plan, du, image_dev(plan, b), want_norm=True)
    gw, hw = oblur.blur_normal(u, b, p, p, bc)
    assert_close(to_host_image(g, rows, cols), gw, what=f"R^*(Ru-b) 2048 {bc}")
    assert abs(float(half) - hw) <= 1e-5 * hw
    # single passes: every CTA of the persistent grid walks several tiles
    assert_close(to_host_image(adj.blur(plan, du), rows, cols), oblur.blur(u, p, p, bc), what=f"R 2048 {bc}")
    assert_close(to_host_image(adj.blur_adjoint(plan, du), rows, cols), oblur.blur_adjoint(u, p, p, bc),
                 what=f"R^* 2048 {bc}")
    assert adj.device_status() == 0


@pytest.mark.parametrize("kr,kc", [(65, 1), (27, 5), (25, 25), (1, 1)])
def test_large_radius_paths_and_identity(adj, kr, kc):
    """Radii above 12 take the runtime-radius kernels, radii up to 12 the
    register-blocked tiles; k = 1 is the identity."""
    pr = random_taps(kr, 3) if kr > 1 else np.array([1.0])
    pc = random_taps(kc, 4) if kc > 1 else np.array([1.0])
    for bc in BCS:
        for rows, cols in [(40, 9), (100, 70), (130, 200)]:
            plan = adj.BlurPlan(rows, cols, pr, pc, bc)
            u = random_vector((rows, cols), 4)
            du = image_dev(plan, u)
            assert_close(to_host_image(adj.blur(plan, du), rows, cols), oblur.blur(u, pr, pc, bc), what="k=65")
            assert_close(to_host_image(adj.blur_adjoint(plan, du), rows, cols),
                         oblur.blur_adjoint(u, pr, pc, bc), what="k=65 adj")
            g = adj.blur_normal(plan, du, None)
            assert_close(to_host_image(g, rows, cols), oblur.blur_normal(u, np.zeros_like(u), pr, pc, bc)[0],
                         what="k=65 normal")


def test_gpu_blur_dot_product(adj):
    pr, pc = random_taps(11, 5), random_taps(7, 6)
    for bc in BCS:
        plan = adj.BlurPlan(200, 150, pr, pc, bc)
        x = image_dev(plan, random_vector((200, 150), 1))
        y = image_dev(plan, random_vector((200, 150), 2))
        lhs = float((adj.blur(plan, x).double() * y.double()).sum())
        rhs = float((x.double() * adj.blur_adjoint(plan, y).double()).sum())
        assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("kr,kc", [(15, 15), (25, 3), (1, 9), (7, 1)])
def test_blur_tma_and_tiled_paths(adj, bc, kr, kc):
    """R and R^* run as persistent TMA-staged passes; R^*(R u - b) with a
    workspace as two such passes, without one as a single fused tiled kernel.
    All against the oracle on shapes spanning several tiles in each direction
    with ragged edges; the device status word stays clear."""
    pr = random_taps(kr, kr + 11) if kr > 1 else np.array([1.0])
    pc = random_taps(kc, kc + 12) if kc > 1 else np.array([1.0])
    for rows, cols in [(200, 300), (131, 257), (64, 128), (13, 600)]:
        plan = adj.BlurPlan(rows, cols, pr, pc, bc)
        u = random_vector((rows, cols), rows + 3 * cols)
        b = random_vector((rows, cols), rows + 5 * cols)
        du, db = image_dev(plan, u), image_dev(plan, b)
        gw, hw = oblur.blur_normal(u, b, pr, pc, bc)
        g1, h1 = adj.blur_normal(plan, du, db, want_norm=True)
        g0 = adj.blur_normal(plan, du, db, scratch=False)
        what = f"{bc} {kr}x{kc} {rows}x{cols}"
        assert_close(to_host_image(g1, rows, cols), gw, what="stream " + what)
        assert_close(to_host_image(g0, rows, cols), gw, what="tiled " + what)
        assert abs(float(h1) - hw) <= 1e-5 * hw
        assert_close(to_host_image(adj.blur(plan, du), rows, cols), oblur.blur(u, pr, pc, bc), what="R " + what)
        assert_close(to_host_image(adj.blur_adjoint(plan, du), rows, cols), oblur.blur_adjoint(u, pr, pc, bc),
                     what="R^* " + what)
    assert adj.device_status() == 0


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("taps", [(15, 3.0, 15, 3.0), (9, 1.5, 5, 1.0), (25, 4.0, 25, 4.0), (3, 0.8, 3, 0.8)],
                         ids=["g15", "g9x5", "g25", "g3"])
def test_normal_palindromic_taps(adj, bc, taps):
    """R^*(R u - b) with Gaussian (palindromic) taps of radii 1 to 12, the
    case in which the symmetric boundary's R^* needs no orientation flips:
    shapes spanning several 32 x 128 tiles with ragged last rows and columns,
    images narrower than a tile and smaller than the PSF, with and without b;
    g element by element and 1/2 ||R u - b||^2 against the oracle."""
    kr, sr, kc, sc = taps
    pr, pc = oblur.gaussian_psf(kr, sr), oblur.gaussian_psf(kc, sc)
    for rows, cols in [(200, 300), (131, 257), (64, 128), (13, 600), (257, 40), (33, 129), (4, 6), (1, 1)]:
        plan = adj.BlurPlan(rows, cols, pr, pc, bc)
        u = random_vector((rows, cols), 3 * rows + cols)
        b = random_vector((rows, cols), 5 * rows + cols)
        du, db = image_dev(plan, u), image_dev(plan, b)
        what = f"{bc} {kr}x{kc} {rows}x{cols}"
        gw, hw = oblur.blur_normal(u, b, pr, pc, bc)
        g, h = adj.blur_normal(plan, du, db, want_norm=True)
        assert_close(to_host_image(g, rows, cols), gw, what="R^*(Ru-b) " + what)
        assert abs(float(h) - hw) <= 1e-5 * hw, what
        g0 = adj.blur_normal(plan, du, None)
        assert_close(to_host_image(g0, rows, cols), oblur.blur_normal(u, np.zeros_like(u), pr, pc, bc)[0],
                     what="R^*R u " + what)
    assert adj.device_status() == 0
