"""conv_adjoint_noalloc: the allocation-free channel gradient.

Callers that must not allocate device memory on their call path (memory owned
by another allocator, loops that cannot take cudaMalloc's device-wide
synchronisation, no allocation after start-up) use this entry point; its
grad_h partial sums live in a fixed array inside the library.  This test calls
it through the C-ABI on every kernel path behind it, twice over with fresh
inputs, and holds each result against conv_adjoint (the workspace entry point)
and against the float64 oracle, with the tolerance of the other parity tests.  It sits in a file of its own that pytest collects last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from synthetic_inputs import channel_problem
from tests.gpu_util import assert_close

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.asarray(a), dtype=torch.float32, device="cuda").contiguous()


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _inputs(B, n, k, seed):
    p = channel_problem(B, n, k, seed=seed)
    r = np.random.default_rng(seed + 1).standard_normal((B, n + k - 1))
    return _dev(p["s_est"]), _dev(p["h_est"]), _dev(r)


def _with_workspace(lib, s, h, r):
    B, n = s.shape
    k = h.shape[1]
    gh = torch.empty(B, k, device="cuda")
    gs = torch.empty(B, n, device="cuda")
    nbytes = lib.adjwt_conv_adjoint_workspace_size(B, n, k)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    off = (-ws.data_ptr()) % 256
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.conv_adjoint(B, n, k, _ptr(s), _ptr(h), _ptr(r), _ptr(gh), _ptr(gs),
                          C.c_void_p(ws.data_ptr() + off), nbytes, stream)
    assert rc == 0, lib.adjwt_last_error()
    return gh, gs


def _no_alloc(lib, s, h, r):
    B, n = s.shape
    k = h.shape[1]
    gh = torch.full((B, k), float("nan"), device="cuda")
    gs = torch.full((B, n), float("nan"), device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.conv_adjoint_noalloc(B, n, k, _ptr(s), _ptr(h), _ptr(r), _ptr(gh), _ptr(gs), stream)
    assert rc == 0, lib.adjwt_last_error()
    return gh, gs


def _oracle_rows(s, h, r, rows):
    from oracle import conv as oconv
    s64, h64, r64 = (t[rows].double().cpu().numpy() for t in (s, h, r))
    return oconv.conv_adjoint(s64, h64, r64)


# Run in this order.  The first case fills the whole fixed scratch (1024 rows x
# 1 chunk x 1024 lags = 2^20 partial sums); every later case is smaller, so a
# partial sum left over from an earlier call in a slot a later call failed to
# write would show up in its grad_h.  The cases take the three kernels behind
# the entry point: the FP32 sliding-window kernel (k <= 1024 outside 49..64),
# the tensor-core kernel (49 <= k <= 64, 4096-sample chunks; the bench's
# k = 64) and the k > 1024 kernel (1024-sample chunks).
CASES = [
    (1024, 3072, 1024, 11),   # FP32 path, whole array
    (64, 65536, 64, 13),      # tensor-core path
    (3, 5000, 2000, 14),      # k > 1024 path
    (7, 3000, 33, 12),        # FP32 path, ragged
    (5, 4099, 49, 15),        # tensor-core path, ragged tail chunk
]


def test_no_alloc_matches_workspace_entry_point_and_oracle_twice():
    from paper_1707_02018_gb300 import _lib
    lib = _lib.load()
    for call in range(2):
        for B, n, k, seed in CASES:
            s, h, r = _inputs(B, n, k, seed + 100 * call)
            want_h, want_s = _with_workspace(lib, s, h, r)
            got_h, got_s = _no_alloc(lib, s, h, r)
            torch.cuda.synchronize()
            what = f"call {call} {B}x{n}x{k}"
            # against the workspace entry point, every element
            assert_close(got_h.cpu().numpy(), want_h.cpu().numpy(), what="grad_h vs conv_adjoint " + what)
            assert_close(got_s.cpu().numpy(), want_s.cpu().numpy(), what="grad_s vs conv_adjoint " + what)
            # against the float64 oracle: every row for the smaller cases,
            # 16 sampled rows of the whole-array case
            rows = np.arange(B) if B * n * k <= 2 ** 28 else np.linspace(0, B - 1, 16).astype(int)
            oh, os_ = _oracle_rows(s, h, r, rows)
            assert_close(got_h[rows].cpu().numpy(), oh, what="grad_h vs oracle " + what)
            assert_close(got_s[rows].cpu().numpy(), os_, what="grad_s vs oracle " + what)


def test_no_alloc_rejects_sizes_beyond_its_scratch():
    from paper_1707_02018_gb300 import _lib
    lib = _lib.load()
    # 1025 rows x 1 chunk x 1024 lags = 1,049,600 partial sums > 2^20: rejected
    # before any pointer is looked at or any kernel is launched
    gh = torch.empty(1025, 1024, device="cuda")
    rc = lib.conv_adjoint_noalloc(1025, 3072, 1024, None, None, None, _ptr(gh), None, None)
    assert rc == -7
    assert b"more than the fixed scratch" in lib.adjwt_last_error()
