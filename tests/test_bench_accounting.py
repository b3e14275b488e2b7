"""The algorithmic byte counts bench.py divides by are those the oracle's own
layout gives (CPU): band sizes of the 5-level CDF 9/7 transform at 2048^2,
the coefficient count C, and the per-step total quoted for the workload."""
import pytest

import bench
from oracle import layout as olayout


@pytest.mark.parametrize("bc,mode", [("per", "per"), ("sym", "sym"), ("zero", "zpd")])
def test_level_sizes_match_oracle_layout(bc, mode):
    got = bench.level_sizes(bench.SIZE, bench.LEVELS, bc)
    want = olayout.level_sizes(bench.SIZE, bench.SIZE, bench.LEVELS, 10, mode)
    assert [(n, m) for n, m in got] == [(N[0], nb[0]) for N, nb in want]


@pytest.mark.parametrize("bc,mode", [("per", "per"), ("sym", "sym"), ("zero", "zpd")])
def test_fista_bytes_from_oracle_counts(bc, mode):
    """W reads C coefficients and writes N^2 pixels plus the intermediate LL
    images (written and read: 2 I); R^*(R u - b) reads u and b and writes g
    (3 N^2); W^* + prox reads the image and the intermediates and reads /
    writes x and y plus the step's g contribution (4 C + N^2 + 2 I)."""
    C = olayout.num_coeffs(bench.SIZE, bench.SIZE, bench.LEVELS, 10, mode)
    sizes = olayout.level_sizes(bench.SIZE, bench.SIZE, bench.LEVELS, 10, mode)
    I = sum(nb[0] * nb[1] for _, nb in sizes[:-1])
    N2 = bench.SIZE ** 2
    fb = bench.fista_bytes(bc)
    assert fb["wt_synth"] == 4 * (C + N2 + 2 * I)
    assert fb["blur_normal"] == 4 * 3 * N2
    assert fb["wt_adjoint_prox"] == 4 * (4 * C + N2 + 2 * I)
    assert fb["total"] == fb["wt_synth"] + fb["blur_normal"] + fb["wt_adjoint_prox"]


def test_step_bytes_total():
    """782.5 MB per step: three FISTA iterations and the channel gradient
    (reads s, h, x; writes grad_s, grad_h of 256 x 65,536 x 64)."""
    B, n, k = 256, 65536, 64
    assert bench.channel_bytes()["total"] == 4 * (2 * B * n + 2 * B * k + B * (n + k - 1))
    assert abs(bench.step_bytes() / 1e6 - 782.5) < 0.1
