"""Autograd wrappers: gradients through W, W^*, R, R^* equal the oracle's
closed-form gradients (the backward of each operator is its exact adjoint)."""
import numpy as np
import pytest
import torch

from oracle import blur as oblur
from oracle import wavelet as owt
from synthetic_inputs import random_taps, random_vector
from tests.gpu_util import assert_close, image_dev, to_host_image

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def adj():
    import paper_1707_02018_gb300 as adj
    adj.lib()
    return adj


@pytest.mark.parametrize("w,mode,bc", [("cdf97", "sym", "sym"), ("db4", "zero", "zero"), ("db2", "per", "per")])
def test_grad_of_data_term_through_W_and_R(adj, w, mode, bc):
    """L(c) = 1/2 ||R W c - b||^2:  dL/dc = W^* R^* (R W c - b)."""
    from paper_1707_02018_gb300 import autograd as ag
    rows, cols, J = 72, 96, 3
    pr, pc = random_taps(7, 3), random_taps(5, 4)  # asymmetric: R^* differs from R
    wt = adj.WtPlan(rows, cols, J, w, mode)
    bl = adj.BlurPlan(rows, cols, pr, pc, bc)
    c = random_vector(wt.logical_size, 5)
    b = random_vector((rows, cols), 6)
    cd = wt.pack(c).requires_grad_(True)
    bd = image_dev(wt, b)
    res = ag.apply_blur(ag.synth(cd, wt), bl) - bd
    loss = 0.5 * (res[:, :cols] ** 2).sum()
    loss.backward()
    u = owt.wt_synth(c, rows, cols, J, w, mode)
    r = oblur.blur(u, pr, pc, bc) - b
    want = owt.wt_adjoint(oblur.blur_adjoint(r, pr, pc, bc), J, w, mode)
    assert_close(wt.unpack(cd.grad).cpu().numpy(), want, what=f"dL/dc {w} {mode}")
    assert abs(float(loss.detach()) - 0.5 * float(np.sum(r * r))) <= 1e-5 * 0.5 * float(np.sum(r * r))


def test_grad_through_adjoints(adj):
    """L(u) = 1/2 ||W^* R^* u||^2:  dL/du = R W W^* R^* u."""
    from paper_1707_02018_gb300 import autograd as ag
    rows, cols, J = 64, 80, 2
    pr = random_taps(9, 7)
    wt = adj.WtPlan(rows, cols, J, "cdf97", "sym")
    bl = adj.BlurPlan(rows, cols, pr, pr[::-1].copy(), "sym")
    u = random_vector((rows, cols), 9)
    ud = image_dev(wt, u).requires_grad_(True)
    z = ag.synth_adjoint(ag.apply_blur_adjoint(ud, bl), wt)
    (0.5 * (z * z).sum()).backward()
    zc = owt.wt_adjoint(oblur.blur_adjoint(u, pr, pr[::-1].copy(), "sym"), J, "cdf97", "sym")
    want = oblur.blur(owt.wt_synth(zc, rows, cols, J, "cdf97", "sym"), pr, pr[::-1].copy(), "sym")
    assert_close(to_host_image(ud.grad, rows, cols), want, what="dL/du")
