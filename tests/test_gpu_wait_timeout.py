"""Failure detection without a GPU fault: the bounded wait used by every
staging and tensor-core completion wait runs out on a barrier that nothing
completes, records ADJWT_ERR_TIMEOUT in the device status word and returns;
the context stays usable."""
import time

import numpy as np
import pytest

from oracle import blur as oblur
from synthetic_inputs import random_vector
from tests.gpu_util import assert_close

pytestmark = pytest.mark.gpu

ADJWT_ERR_TIMEOUT = -8


@pytest.fixture(scope="module")
def adj():
    import paper_1707_02018_gb300 as adj
    adj.lib()
    return adj


def test_bounded_wait_runs_out_and_the_context_stays_usable(adj):
    adj.device_status(clear=True)
    adj.wait_selftest(True)                      # the barrier completes: no timeout
    assert adj.device_status() == 0
    t0 = time.perf_counter()
    adj.wait_selftest(False)                     # nothing completes it
    status = adj.device_status(clear=True)       # synchronises
    elapsed = time.perf_counter() - t0
    assert status == ADJWT_ERR_TIMEOUT
    assert 0.1 < elapsed < 60.0, elapsed         # it waited up to its limit, then returned
    assert adj.device_status() == 0              # cleared
    # the context still computes: one blur pass against the oracle
    rows, cols = 40, 56
    p = oblur.gaussian_psf(7, 1.3)
    plan = adj.BlurPlan(rows, cols, p, p, "sym")
    u = random_vector((rows, cols), 3)
    out = adj.blur(plan, plan.image(u))
    assert_close(out[:, :cols].double().cpu().numpy(), oblur.blur(u, p, p, "sym"), what="blur after a timeout")
    assert adj.device_status() == 0
