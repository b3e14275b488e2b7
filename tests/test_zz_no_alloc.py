"""conv_adjoint_noalloc: the allocation-free channel gradient.

Callers that must not allocate device memory on their call path (memory owned
by another allocator, loops that cannot take cudaMalloc's device-wide
synchronisation, no allocation after start-up) use this entry point; its
grad_h partial sums live in a fixed array inside the library.  This test calls
it through the C-ABI twice in a row, on different inputs, and holds each result
against conv_adjoint (the workspace entry point) with the tolerance of the
other parity tests.  It sits in a file of its own that pytest collects last.
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


def test_no_alloc_matches_workspace_entry_point_twice():
    from paper_1707_02018_gb300 import _lib
    lib = _lib.load()
    # the first call fills the whole fixed scratch (1024 rows x 1 chunk x 1024
    # lags = 2^20 partial sums); the second is smaller, so a partial sum left over
    # from the first call in a slot the second call failed to write would show
    # up in its grad_h
    cases = [(1024, 3072, 1024, 11), (7, 3000, 33, 12)]
    for B, n, k, seed in cases:
        s, h, r = _inputs(B, n, k, seed)
        want_h, want_s = _with_workspace(lib, s, h, r)
        got_h, got_s = _no_alloc(lib, s, h, r)
        torch.cuda.synchronize()
        assert_close(got_h.cpu().numpy(), want_h.cpu().numpy(), what=f"grad_h {B}x{n}x{k}")
        assert_close(got_s.cpu().numpy(), want_s.cpu().numpy(), what=f"grad_s {B}x{n}x{k}")


def test_no_alloc_rejects_sizes_beyond_its_scratch():
    from paper_1707_02018_gb300 import _lib
    lib = _lib.load()
    # 1025 rows x 1 chunk x 1024 lags = 1,049,600 partial sums > 2^20: rejected
    # before any pointer is looked at or any kernel is launched
    gh = torch.empty(1025, 1024, device="cuda")
    rc = lib.conv_adjoint_noalloc(1025, 3072, 1024, None, None, None, _ptr(gh), None, None)
    assert rc == -7
    assert b"exceeds the fixed scratch" in lib.adjwt_last_error()
