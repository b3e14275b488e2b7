"""Host-side checks of the C-ABI library (no GPU needed, no kernel launched).

* libadjwt.so loads and exports every function include/adjwt.h declares;
* plan layouts (sizes, offsets, pitches) match the oracle's band sizes;
* the device path's own filter derivation matches the oracle's taps;
* argument validation rejects bad calls before anything reaches the device.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest
import torch

from oracle import filters as ofilters
from oracle import layout as olayout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "adjwt.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1707_02018_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_1707_02018_gb300 import build_ext
        build_ext.build()
    return _lib.load()


def declared_functions():
    import glob
    text = "".join(open(h).read() for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|size_t|char)\s*\*?\s*(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in ["wt_synth", "wt_synth_adjoint", "blur", "blur_adjoint", "conv_adjoint", "fista_step"]:
        assert n in names
    for n in names:
        assert hasattr(lib, n), f"libadjwt.so does not export {n}"
    from paper_1707_02018_gb300._lib import PROTOTYPES
    assert set(PROTOTYPES) == set(names)


def _plan(lib, rows, cols, levels, w, bc):
    h = C.c_void_p()
    rc = lib.adjwt_wt_plan_create(C.byref(h), rows, cols, levels, w, bc)
    return rc, h


WAV = {"haar": 0, "db2": 1, "db4": 2, "cdf97": 3}


@pytest.mark.parametrize("w", list(WAV))
@pytest.mark.parametrize("bc,mode", [(0, "zero"), (3, "per")])
@pytest.mark.parametrize("rows,cols,J", [(2048, 2048, 5), (256, 256, 3), (37, 53, 2), (64, 32, 4), (1, 1, 1)])
def test_layout_matches_oracle(lib, w, bc, mode, rows, cols, J):
    if mode == "per" and (rows % 2 ** J or cols % 2 ** J):
        rc, _ = _plan(lib, rows, cols, J, WAV[w], bc)
        assert rc == -2                                     # ADJWT_ERR_SHAPE
        return
    rc, h = _plan(lib, rows, cols, J, WAV[w], bc)
    assert rc == 0, lib.adjwt_last_error()
    nb = 3 * J + 1
    nc = C.c_int64()
    offs = (C.c_int64 * nb)()
    br, bcl, bp = (C.c_int * nb)(), (C.c_int * nb)(), (C.c_int * nb)()
    ip = C.c_int()
    assert lib.adjwt_wt_layout(h, C.byref(nc), offs, br, bcl, bp, C.byref(ip)) == 0
    L = ofilters.filter_bank(w).L
    sizes = olayout.level_sizes(rows, cols, J, L, mode)
    want = [sizes[-1][1]] + [sizes[j - 1][1] for j in range(J, 0, -1) for _ in range(3)]
    assert [(br[i], bcl[i]) for i in range(nb)] == want
    pos = 0
    for i in range(nb):
        assert offs[i] == pos and bp[i] % 4 == 0 and bp[i] >= bcl[i] and bp[i] - bcl[i] < 4
        pos += br[i] * bp[i]
    assert nc.value == pos
    assert ip.value % 4 == 0 and ip.value - cols < 4
    assert sum(r * c for r, c in want) == olayout.num_coeffs(rows, cols, J, L, mode)
    lib.adjwt_wt_plan_destroy(h)


@pytest.mark.parametrize("w", list(WAV))
def test_device_path_filters_match_oracle(lib, w):
    rc, h = _plan(lib, 64, 64, 1, WAV[w], 0)
    assert rc == 0
    arrs = [(C.c_double * 10)() for _ in range(4)]
    L = C.c_int()
    assert lib.adjwt_wt_filters(h, *arrs, C.byref(L)) == 0
    fb = ofilters.filter_bank(w)
    assert L.value == fb.L
    for got, want in zip(arrs, (fb.dec_lo, fb.dec_hi, fb.rec_lo, fb.rec_hi)):
        assert np.abs(np.array(list(got)[:fb.L]) - want).max() < 1e-13
    lib.adjwt_wt_plan_destroy(h)


def test_plan_argument_errors(lib):
    h = C.c_void_p()
    assert lib.adjwt_wt_plan_create(C.byref(h), 8, 8, 1, 7, 0) == -1       # unknown wavelet
    assert lib.adjwt_wt_plan_create(C.byref(h), 8, 8, 1, 0, 9) == -1       # unknown bc
    assert lib.adjwt_wt_plan_create(C.byref(h), 0, 8, 1, 0, 0) == -2       # empty image
    assert lib.adjwt_wt_plan_create(C.byref(h), 8, 8, 0, 0, 0) == -2       # no level
    assert lib.adjwt_wt_plan_create(C.byref(h), 12, 8, 3, 0, 3) == -2      # PER needs 2^J | size
    assert lib.adjwt_wt_plan_create(None, 8, 8, 1, 0, 0) == -1
    taps = (C.c_double * 4)(0.25, 0.25, 0.25, 0.25)
    assert lib.adjwt_blur_plan_create(C.byref(h), 8, 8, taps, 4, taps, 3, 1) == -1   # even length
    assert lib.adjwt_blur_plan_create(C.byref(h), 8, 8, taps, 3, taps, 3, 2) == -1   # PPD not a blur bc
    assert b"odd" in lib.adjwt_last_error() or len(lib.adjwt_last_error()) > 0


@pytest.mark.skipif(torch.cuda.is_available(), reason="fake-pointer validation runs on the host only")
def test_call_validation_before_launch(lib):
    """Calls that must fail in validation (fake addresses are never dereferenced)."""
    rc, h = _plan(lib, 16, 16, 1, 1, 0)
    assert rc == 0
    ws_need = lib.adjwt_wt_workspace_size(h)
    assert ws_need > 0
    a, b, ws = 0x10000000, 0x20000000, 0x30000000
    assert lib.wt_synth(h, None, b, ws, ws_need, None) == -1
    assert lib.wt_synth(h, a + 4, b, ws, ws_need, None) == -3              # misaligned
    assert lib.wt_synth(h, a, a + 16, ws, ws_need, None) == -4             # aliasing
    assert lib.wt_synth(h, a, b, None, ws_need, None) == -7                # no workspace
    assert lib.wt_synth(h, a, b, ws + 16, ws_need, None) == -7             # misaligned workspace
    assert lib.wt_synth(h, a, b, ws, ws_need - 1, None) == -7              # small workspace
    assert lib.wt_synth(None, a, b, ws, ws_need, None) == -1
    assert lib.conv_adjoint(-1, 5, 3, a, b, ws, None, None, None, 0, None) == -2
    assert lib.conv_adjoint(4, 0, 3, a, b, ws, None, None, None, 0, None) == -2
    assert lib.conv_adjoint(0, 5, 3, None, None, None, None, None, None, 0, None) == 0   # empty batch
    assert lib.conv_adjoint(2, 5, 3, a, b, ws, a, None, None, 0, None) == -4  # grad_h over s
    lib.adjwt_wt_plan_destroy(h)


def test_conv_adjoint_noalloc_validation(lib):
    """The allocation-free channel gradient checks sizes, pointers and aliasing
    on the host before it looks up its fixed array or launches anything."""
    a, b, c = 0x10000000, 0x20000000, 0x30000000
    f = lib.conv_adjoint_noalloc
    assert f(-1, 5, 3, a, b, c, None, None, None) == -2                 # negative batch
    assert f(4, 0, 3, a, b, c, None, None, None) == -2                  # empty rows
    assert f(4, 5, 0, a, b, c, None, None, None) == -2                  # no taps
    assert f(65536, 5, 3, a, b, c, None, None, None) == -2              # batch above 65535
    assert f(0, 5, 3, None, None, None, None, None, None) == 0          # empty batch: nothing to do
    assert f(2, 5, 3, None, None, None, None, None, None) == 0          # no output requested
    # 1025 rows x 1 chunk (3072 samples) x 1024 lags = 1,049,600 partial sums > 2^20
    assert f(1025, 3072, 1024, None, None, None, c, None, None) == -7
    assert b"more than the fixed scratch" in lib.adjwt_last_error()
    # 1024 rows fit exactly (2^20); the call then fails only on its NULL inputs
    assert f(1024, 3072, 1024, None, None, None, c, None, None) == -1
    # 17 chunks of 4032 samples at k = 64: 1000 x 17 x 64 = 1,088,000 > 2^20
    assert f(1000, 65536, 64, a, b, c, 0x40000000, None, None) == -7
    # without grad_h no scratch is used, so the same sizes pass the size check
    assert f(1000, 65536, 64, a, b, c, None, 0x40000000 + 4, None) == -3   # misaligned grad_s
    assert f(2, 5, 3, a, b, c, a, None, None) == -4                     # grad_h over s
    assert f(2, 5, 3, a, b, c, c + 16, None, None) == -4                # grad_h over r
    assert f(2, 5, 3, a, b, c, None, c, None) == -4                     # grad_s over r
    assert f(2, 5, 3, a, b, c, None, b, None) == -4                     # grad_s over h


def test_workspace_sizes(lib):
    # one partial grad_h per (row, chunk) with chunks of 32*floor((4097-k)/32) = 4032 samples at k = 64
    assert lib.adjwt_conv_adjoint_workspace_size(256, 65536, 64) >= 256 * 17 * 64 * 4
    assert lib.adjwt_conv_adjoint_workspace_size(2, 10000, 2000) >= 2 * 10 * 2000 * 4
    assert lib.adjwt_conv_gradient_workspace_size(2, 10000, 2000) >= 2 * 10 * 2000 * 4 + 2 * 11999 * 4
    assert lib.adjwt_conv_adjoint_workspace_size(0, 10, 3) == 0
    rc, h = _plan(lib, 2048, 2048, 5, 3, 3)
    assert rc == 0
    assert lib.adjwt_wt_workspace_size(h) >= (1024 * 1024 + 512 * 512) * 4
    lib.adjwt_wt_plan_destroy(h)


def test_level_implementation_switches(lib):
    """The per-level TMA / tiled switch (host logic; no GPU needed): the size
    rule gives level 1 of a 2048^2 PER plan to the TMA kernels, small levels
    never; the switch and its argument checks."""
    h = C.c_void_p()
    assert lib.adjwt_wt_plan_create(C.byref(h), 2048, 2048, 5, 1, 3) == 0   # db2, PER
    uses = C.c_int()
    try:
        for op in (0, 1, 2):
            assert lib.adjwt_wt_plan_uses_tma(h, op, 1, C.byref(uses)) == 0 and uses.value == 1
            assert lib.adjwt_wt_plan_uses_tma(h, op, 5, C.byref(uses)) == 0 and uses.value == 0
            assert lib.adjwt_wt_plan_set_tma(h, op, 1, 0) == 0
            assert lib.adjwt_wt_plan_uses_tma(h, op, 1, C.byref(uses)) == 0 and uses.value == 0
            assert lib.adjwt_wt_plan_set_tma(h, op, 1, 1) == 0
            assert lib.adjwt_wt_plan_uses_tma(h, op, 1, C.byref(uses)) == 0 and uses.value == 1
        assert lib.adjwt_wt_plan_set_tma(h, 0, 6, 0) == -2     # level out of range
        assert lib.adjwt_wt_plan_set_tma(h, 0, 0, 0) == -2
        assert lib.adjwt_wt_plan_set_tma(h, 3, 1, 0) == -1     # unknown operator
        assert lib.adjwt_wt_plan_uses_tma(h, 0, 1, None) == -1
        assert lib.adjwt_wt_plan_autotune(h, 0, None, None) == -1   # reps outside 1..1000
    finally:
        lib.adjwt_wt_plan_destroy(h)


def test_differentiation_entry_validation(lib):
    """The differentiation entries reject bad arguments before any launch."""
    assert lib.adjwt_axpby(-1, 1.0, None, 1.0, None, None, None) == -2
    assert lib.adjwt_axpby(0, 1.0, None, 1.0, None, None, None) == 0        # nothing to do
    assert lib.adjwt_axpby(4, 1.0, None, 1.0, None, None, None) == -1       # NULL buffers
    assert lib.adjwt_dot(2, 5, 4, None, None, None, None, 0, None) == -2      # pitch < cols
    assert lib.adjwt_dot(1, 4, 4, None, None, None, None, 0, None) == -1      # NULL buffers
    fake = C.c_void_p(256)                                                   # never dereferenced
    assert lib.adjwt_dot(1, 4, 4, fake, fake, fake, None, 0, None) == -7     # no workspace
    assert lib.adjwt_dot(1, 4, 4, fake, fake, fake, fake, 8, None) == -7     # workspace too small
    assert lib.fista_prox_vjp(-1, None, None, None, None, None, 0, None) == -2
    assert lib.fista_prox_vjp(4, fake, fake, fake, fake, None, 0, None) == -7
    assert lib.adjwt_reduce_workspace_size() >= 8


@pytest.mark.skipif(torch.cuda.is_available(), reason="fake-pointer validation runs on the host only")
def test_vjp_step_validation(lib):
    """fista_vjp_step rejects bad problems, pointers and workspaces before any
    launch; its workspace holds at least the seven images and three coefficient
    vectors it uses.  Fake device addresses are never dereferenced; a zeroed
    host buffer stands in for a blur plan of an empty image (blur plans hold
    device taps and cannot be created without a GPU)."""
    from paper_1707_02018_gb300._lib import FistaProblem
    rc, wt = _plan(lib, 64, 48, 2, 1, 3)   # db2, PER: no boundary tables to upload
    assert rc == 0
    zero_plan = (C.c_char * 4096)()
    R = C.cast(zero_plan, C.c_void_p)
    a, ws = 0x10000000, 0x30000000
    prob = FistaProblem(wt, R, a, 0.01, 2.0, 0)
    try:
        need = lib.adjwt_fista_vjp_workspace_size(C.byref(prob))
        assert need >= 7 * 64 * 48 * 4 + 3 * 64 * 48 * 4
        assert lib.adjwt_fista_vjp_workspace_size(None) == 0

        def call(x=a, dsig=None, d1=None, d2=None, w=ws, nbytes=need):
            return lib.fista_vjp_step(C.byref(prob), d1, d2, x, a, 0.5, a, a, None, a, dsig, w, nbytes, None)

        assert lib.fista_vjp_step(None, None, None, a, a, 0.5, a, a, None, a, None, ws, need, None) == -1
        assert call(x=None) == -1                     # NULL x_next
        assert call(x=a + 4) == -3                    # misaligned vector
        assert call(dsig=a) == -1                     # dsigma without the dR plans
        assert call(w=None) == -7                     # no workspace
        assert call(w=ws + 16) == -7                  # misaligned workspace
        assert call(nbytes=need - 1) == -7            # small workspace
        assert call() == -2                           # blur plan of another (empty) image
        prob.gradient = 1
        assert call() == -1                           # W^dagger iteration: not differentiable
        prob.gradient, prob.lipschitz = 0, 0.0
        assert call() == -1                           # L = 0
        prob.lipschitz, prob.blur = 2.0, None
        assert call() == -1                           # no blur plan
    finally:
        lib.adjwt_wt_plan_destroy(wt)


@pytest.mark.skipif(torch.cuda.is_available(), reason="fake-pointer validation runs on the host only")
def test_cnn_entry_validation(lib):
    """The learned-warm-start entries reject bad sizes, pointers and
    workspaces before any launch (fake addresses are never dereferenced)."""
    a = 0x10000000
    assert lib.adjwt_cnn_param_count() == 56097
    assert lib.adjwt_cnn_packed_bytes() == 6 * 2 * 18 * 1024
    assert lib.adjwt_cnn_activation_bytes(2, 8, 8) == 7 * 2 * 8 * 8 * 32 * 2
    assert lib.adjwt_cnn_activation_bytes(-1, 8, 8) == 0
    assert lib.adjwt_cnn_workspace_size(2, 8, 8) >= 2 * 8 * 8 * (4 + 2 * 64)
    assert lib.cnn_forward(-1, 8, 8, a, 8, a, a, a, a, None) == -2
    assert lib.cnn_forward(0, 8, 8, None, 8, None, None, None, None, None) == 0     # empty batch
    assert lib.cnn_forward(1, 8, 8, a, 4, a, a, a, a, None) == -2                    # pitch < cols
    assert lib.cnn_forward(1, 8, 8, a, 8, None, a, a, a, None) == -1                 # no params
    assert lib.cnn_forward(1, 8, 8, a + 4, 8, a, a, a, a, None) == -3                # misaligned b
    assert lib.cnn_backward(1, 8, 8, a, a, a, 8, a, a, a, a, a, None, 0, None) == -7  # no workspace
    assert lib.cnn_backward(1, 8, 8, a, a, a, 8, a, a, a, a, a, a + 16, 1 << 30, None) == -7  # misaligned
    assert lib.cnn_adam(10, a, a, a, a, 0, 1e-3, 0.9, 0.999, 1e-8, None) == -1      # step 0
    assert lib.cnn_adam(10, a, a, a, a, 1, 1e-3, 1.0, 0.999, 1e-8, None) == -1      # beta1 = 1
    assert lib.cnn_adam(10, a, a, a, a, 1, 1e-3, 0.9, 0.999, 0.0, None) == -1       # eps = 0
    assert lib.cnn_adam(0, None, None, None, None, 1, 1e-3, 0.9, 0.999, 1e-8, None) == 0
    assert lib.cnn_conv32(1, 4, 4, a, a, None, 1, None, a + 16, None) == -4          # out overlaps in
    assert lib.cnn_conv32(1, 4, 4, a, None, None, 1, None, a + 4096, None) == -1
    assert lib.cnn_conv32_wgrad(1, 4, 4, a, a, a, a, None, 0, None) == -7
    assert lib.cnn_pack(None, a, None) == -1


def test_missing_library_fails_loudly(tmp_path):
    """Without libadjwt.so the binding raises: there is no CPU fallback."""
    import subprocess
    import sys
    code = ("from paper_1707_02018_gb300 import _lib\n"
            "_lib._lib = None\n"
            "try:\n"
            f"    _lib.load({str(tmp_path / 'libadjwt.so')!r})\n"
            "except RuntimeError as e:\n"
            "    print('raised', 'no CPU fallback' in str(e))\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert out.stdout.strip() == "raised True", out.stdout + out.stderr


def test_fista_momentum_matches_oracle(lib):
    """The momentum fista_step applies (host routine, no device work) follows
    the oracle's t-update; beta is its float32 rounding."""
    from oracle import fista as ofista
    t = 1.0
    for _ in range(50):
        t1, beta = C.c_double(), C.c_float()
        assert lib.adjwt_fista_momentum(t, C.byref(t1), C.byref(beta)) == 0
        want_t1 = ofista.t_next(t)
        assert abs(t1.value - want_t1) <= 1e-15 * want_t1
        assert beta.value == np.float32((t - 1.0) / want_t1)
        t = t1.value
    assert lib.adjwt_fista_momentum(0.5, C.byref(C.c_double()), C.byref(C.c_float())) == -1
    assert lib.adjwt_fista_momentum(float("nan"), C.byref(C.c_double()), C.byref(C.c_float())) == -1
    assert lib.adjwt_fista_momentum(1.0, None, C.byref(C.c_float())) == -1


def test_level_chain_range(lib):
    """Which levels run as one level-chain launch (plans without 1/c tables,
    so nothing touches a device): 2048^2 CDF 9/7 J=5 chains 2..5 under ZERO
    (level 1 is the TMA kernels'), and under PER W chains 4..5 (levels 1-3 are
    whole TMA levels) while W^* chains 2..5;
    a small ZERO image chains every level; one level has no chain.  The chain
    is off until switched on."""
    def starts(h):
        out = []
        for op in range(3):
            v = C.c_int(-1)
            assert lib.adjwt_wt_plan_chain_start(h, op, C.byref(v)) == 0
            out.append(v.value)
        return out
    for (rows, J, bc, want) in [(2048, 5, 0, [2, 2, 2]), (2048, 5, 3, [4, 2, 2]), (256, 3, 0, [1, 1, 1]),
                                (256, 1, 0, [0, 0, 0])]:
        rc, h = _plan(lib, rows, rows, J, WAV["cdf97"], bc)
        assert rc == 0, lib.adjwt_last_error()
        assert starts(h) == [0, 0, 0]                       # off by default
        assert lib.adjwt_wt_plan_set_level_chain(h, 1) == 0
        assert starts(h) == want, (rows, J, bc)
        assert lib.adjwt_wt_plan_set_level_chain(h, 0) == 0
        assert starts(h) == [0, 0, 0]
        lib.adjwt_wt_plan_destroy(h)
    assert lib.adjwt_wt_plan_chain_start(None, 0, C.byref(C.c_int())) == -1
    rc, h = _plan(lib, 64, 64, 2, WAV["db2"], 0)
    assert lib.adjwt_wt_plan_chain_start(h, 3, C.byref(C.c_int())) == -1
    lib.adjwt_wt_plan_destroy(h)


def test_trace_level_validation(lib):
    """adjwt_trace_set_level takes 1 (every kernel) or 2 (whole operator calls)
    and rejects anything else before any device work."""
    assert lib.adjwt_trace_set_level(0) == -1
    assert lib.adjwt_trace_set_level(3) == -1
    assert lib.adjwt_trace_set_level(2) == 0
    assert lib.adjwt_trace_set_level(1) == 0


def test_tma_cta_cap_validation(lib):
    """adjwt_wt_plan_set_tma_ctas / adjwt_wt_plan_tma_ctas: caps 0..3 per op and
    level are stored and read back; bad op, level or cap are rejected on the host."""
    rc, h = _plan(lib, 64, 64, 3, WAV["db2"], 3)   # PER: no boundary tables to upload
    assert rc == 0
    try:
        v = C.c_int(-1)
        assert lib.adjwt_wt_plan_tma_ctas(h, 2, 1, C.byref(v)) == 0 and v.value == 0
        assert lib.adjwt_wt_plan_set_tma_ctas(h, 2, 1, 1) == 0
        assert lib.adjwt_wt_plan_tma_ctas(h, 2, 1, C.byref(v)) == 0 and v.value == 1
        assert lib.adjwt_wt_plan_set_tma_ctas(h, 3, 1, 1) == -1       # op
        assert lib.adjwt_wt_plan_set_tma_ctas(h, 0, 4, 1) == -2       # level (SHAPE)
        assert lib.adjwt_wt_plan_set_tma_ctas(h, 0, 1, 4) == -1       # cap
        assert lib.adjwt_wt_plan_tma_ctas(h, 0, 1, None) == -1
    finally:
        lib.adjwt_wt_plan_destroy(h)


def test_fista_batch_entry_validation(lib):
    """The batched engine's entry points reject bad calls on the host, before
    any device memory is touched: NULL handles and arrays, counts outside
    1..65535, a problem without plans, and plans of different images (a
    zeroed host buffer stands in for a blur plan of an empty image; fake
    device addresses are never dereferenced)."""
    from paper_1707_02018_gb300._lib import FistaProblem
    rc, wt = _plan(lib, 64, 48, 2, 1, 3)   # db2, PER: no boundary tables to upload
    assert rc == 0
    zero_plan = (C.c_char * 4096)()
    R = C.cast(zero_plan, C.c_void_p)
    a, ws = 0x10000000, 0x30000000
    probs = (FistaProblem * 2)(FistaProblem(wt, R, a, 0.01, 2.0, 0), FistaProblem(wt, R, a, 0.01, 2.0, 0))
    xs = (C.c_void_p * 2)(a, a + 4096)
    ys = (C.c_void_p * 2)(a + 8192, a + 12288)
    h = C.c_void_p(0x1234)
    try:
        assert lib.adjwt_fista_batch_workspace_size(0, probs) == 0
        assert lib.adjwt_fista_batch_workspace_size(2, None) == 0
        create = lib.adjwt_fista_batch_create
        assert create(None, 2, probs, xs, ys, ws, 1 << 30) == -1             # no output handle
        assert create(C.byref(h), 0, probs, xs, ys, ws, 1 << 30) == -1       # empty batch
        assert h.value is None                                                # cleared on failure
        assert create(C.byref(h), 65536, probs, xs, ys, ws, 1 << 30) == -1   # too many problems
        assert create(C.byref(h), 2, None, xs, ys, ws, 1 << 30) == -1        # no problems
        assert create(C.byref(h), 2, probs, None, ys, ws, 1 << 30) == -1     # no x array
        assert create(C.byref(h), 2, probs, xs, None, ws, 1 << 30) == -1     # no y array
        assert create(C.byref(h), 2, probs, xs, ys, ws, 1 << 30) == -2       # blur plan of another image
        probs[1].wt = None
        assert lib.adjwt_fista_batch_workspace_size(2, probs) == 0
        probs[0].blur = None
        assert create(C.byref(h), 2, probs, xs, ys, ws, 1 << 30) == -1      # problem 0 without a blur plan
        assert h.value is None
        n = C.c_int()
        assert lib.adjwt_fista_batch_info(None, C.byref(n), None, None) == -1
        assert lib.adjwt_fista_batch_run(None, 1, None) == -1
        assert lib.adjwt_fista_batch_objective(None, a, None) == -1
        assert lib.adjwt_fista_batch_reset(None, None) == -1
        assert lib.adjwt_fista_batch_set_iteration(None, 3, None) == -1
        assert lib.adjwt_fista_batch_wait_selftest(None, None) == -1
        lib.adjwt_fista_batch_destroy(None)
    finally:
        lib.adjwt_wt_plan_destroy(wt)


@pytest.mark.skipif(torch.cuda.is_available(), reason="fake-pointer validation runs on the host only")
def test_more_entry_validation(lib):
    """Operators, FISTA helpers and the trace pool reject bad calls before any
    launch: NULL plans and problems, shapes out of range, a non-finite or
    negative threshold, trace indices outside the records.  Fake device
    addresses are never dereferenced."""
    from paper_1707_02018_gb300._lib import FistaProblem
    a, ws = 0x10000000, 0x30000000
    assert lib.adjwt_version() == 1
    assert lib.blur_normal(None, a, a, a, None, None, 0, None) == -1
    assert lib.wt_analysis(None, a, a, ws, 1 << 20, None) == -1
    assert lib.conv_residual(-1, 10, 3, a, a, a, a, None) == -2
    assert lib.conv_residual(1, 0, 3, a, a, a, a, None) == -2
    assert lib.conv_residual(70000, 10, 3, a, a, a, a, None) == -2
    assert lib.conv_residual(0, 10, 3, None, None, None, None, None) == 0   # empty batch: nothing to do
    assert lib.bce_gradient(0, 10, 3, a, a, a, 0.1, 0.5, a, a, ws, 1 << 20, None) == -2
    assert lib.bce_gradient(2, 10, 5000, a, a, a, 0.1, 0.5, a, a, ws, 1 << 20, None) == -2   # k above 4096
    assert lib.bce_gradient(2, 10, 3, a, a, a, 0.1, 0.0, a, a, ws, 1 << 20, None) == -1      # delta = 0
    assert lib.bce_gradient(2, 10, 3, a, a, a, -1.0, 0.5, a, a, ws, 1 << 20, None) == -1     # lambda_tv < 0
    assert lib.adjwt_soft_threshold(-1, a, 0.1, a, None) == -2
    assert lib.adjwt_soft_threshold(0, None, 0.1, None, None) == 0
    assert lib.adjwt_soft_threshold(8, None, 0.1, a, None) == -1
    assert lib.adjwt_soft_threshold(8, a, -0.5, a, None) == -1
    assert lib.adjwt_soft_threshold(8, a, float("nan"), a, None) == -1
    out = C.c_double()
    assert lib.fista_step_device(None, a, a, ws, 1 << 20, None, None) == -1
    assert lib.adjwt_fista_objective(None, a, ws, 1 << 20, C.byref(out), None) == -1
    assert lib.adjwt_fista_lipschitz(None, a, 5, ws, 1 << 20, C.byref(out), None) == -1
    assert lib.adjwt_fista_device_reset(None, ws, 1 << 20, None) == -1
    rc, wt = _plan(lib, 64, 48, 2, 1, 3)   # db2, PER
    assert rc == 0
    zero_plan = (C.c_char * 4096)()
    try:
        prob = FistaProblem(wt, C.cast(zero_plan, C.c_void_p), a, 0.01, 2.0, 0)
        assert lib.fista_step_device(C.byref(prob), a, a, ws, 1 << 20, None, None) == -2        # plans of two images
        assert lib.adjwt_fista_lipschitz(C.byref(prob), a, 5, ws, 1 << 20, C.byref(out), None) == -2
        assert lib.adjwt_fista_device_reset(C.byref(prob), ws, 1 << 20, None) == -2
        assert lib.wt_analysis(wt, None, a, ws, 1 << 20, None) == -1                            # NULL image
    finally:
        lib.adjwt_wt_plan_destroy(wt)
    n = lib.adjwt_trace_count()
    assert n >= 0
    name, tag, ms = C.c_char_p(), C.c_int(), C.c_float()
    assert lib.adjwt_trace_get(-1, C.byref(name), C.byref(tag), C.byref(ms)) == -1
    assert lib.adjwt_trace_get(n, C.byref(name), C.byref(tag), C.byref(ms)) == -1
    assert lib.adjwt_trace_span(0, n, C.byref(ms)) == -1
    assert lib.adjwt_trace_span(0, 0, None) == -1
