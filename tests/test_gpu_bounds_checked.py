"""The bounds-checked build (-DADJWT_BOUNDS_CHECK): every checked global
access of the tile bodies (wavelet levels, the fused blur tile, the TMA
kernels' border completions) is tested against its buffer's extent, and a
violation is recorded in the device status word as ADJWT_ERR_BOUNDS instead
of being performed.  The build runs the parity cases of the wavelet, blur,
FISTA and batched-engine paths in a child process; every result matches the
oracle and no violation is recorded."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_records_no_violation():
    from paper_1707_02018_gb300 import build_ext
    lib = build_ext.build(checked=True)
    env = dict(os.environ, ADJWT_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_checked_child.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert res["status"] == {"wavelet": 0, "blur": 0, "fista": 0}, res["status"]
    for what, err in res["errors"].items():
        tol = 1e-4 if ("FISTA" in what or "batch" in what) else 1e-5
        assert err <= tol, (what, err)
