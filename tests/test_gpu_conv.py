"""Parity of the CUDA blind-channel gradients with the float64 oracle (Sec. II, Eq. 5)."""
import numpy as np
import pytest
import torch

from oracle import conv as oconv
from synthetic_inputs import channel_problem, random_vector
from tests.gpu_util import assert_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def adj():
    import paper_1707_02018_gb300 as adj
    adj.lib()
    return adj


def dev(a):
    return torch.as_tensor(np.asarray(a), dtype=torch.float32, device="cuda").contiguous()


def test_paper_k3_n5_exact(adj):
    """Integer data of the K = 3, N = 5 example: float32 sums are exact."""
    h = np.array([[2.0, -1.0, 3.0]])
    s = np.array([[1.0, 4.0, -2.0, 5.0, 3.0]])
    r = np.array([[1.0, -2.0, 0.0, 7.0, 2.0, -1.0, 4.0]])
    gh, gs = adj.conv_adjoint(dev(s), dev(h), dev(r))
    wh, ws = oconv.conv_adjoint(s, h, r)
    assert np.array_equal(gh.cpu().numpy(), wh) and np.array_equal(gs.cpu().numpy(), ws)
    x = np.array([[0.0, 1.0, 0.0, 0.0, 2.0, 0.0, 1.0]])
    res = adj.conv_residual(dev(h), dev(s), dev(x))
    assert np.array_equal(res.cpu().numpy(), oconv.conv_full(h, s) - x)


@pytest.mark.parametrize("B,n,k", [(3, 5, 3), (2, 1, 1), (4, 1000, 64), (2, 1025, 7), (1, 3, 9), (5, 3000, 300),
                                   (2, 2048, 257), (1, 4097, 1), (2, 8129, 64), (3, 16333, 57), (1, 20000, 49),
                                   (2, 30, 64)])
def test_conv_parity(adj, B, n, k):
    p = channel_problem(B, n, k, seed=B * 1000 + n + k)
    x = oconv.conv_full(p["h"], p["s"]) + p["noise"]
    r = oconv.conv_full(p["h_est"], p["s_est"]) - x
    gh, gs = adj.conv_adjoint(dev(p["s_est"]), dev(p["h_est"]), dev(r))
    wh, ws = oconv.conv_adjoint(p["s_est"], p["h_est"], r)
    assert_close(gh.cpu().numpy(), wh, what=f"grad_h {B}x{n}x{k}")
    assert_close(gs.cpu().numpy(), ws, what=f"grad_s {B}x{n}x{k}")
    rr = adj.conv_residual(dev(p["h_est"]), dev(p["s_est"]), dev(x))
    assert_close(rr.cpu().numpy(), r, what=f"residual {B}x{n}x{k}")


@pytest.mark.parametrize("B,n,k", [(3, 5, 3), (2, 1, 1), (4, 1000, 64), (2, 4033, 64), (2, 8065, 64),
                                   (1, 3, 9), (3, 3000, 300), (2, 5000, 1024), (2, 3000, 1025), (1, 7000, 17),
                                   (2, 8128, 64), (2, 8129, 64), (3, 16333, 57), (1, 24389, 49), (2, 63, 64),
                                   (1, 1, 64), (2, 9000, 48), (2, 9000, 65)])
def test_conv_gradient_fused_parity(adj, B, n, k):
    """r = h * s - x and both gradients in one call.  49 <= k <= 64 runs on
    the tensor-core kernel (chunks of 8128 samples: edges at 8128, 16256 and
    a ragged tail); k = 48 and 65 sit just outside it on the register-blocked
    kernel (chunk edges at 4032 / 8064 for k = 64 there); k = 1025 takes the
    two-kernel path with r in the workspace."""
    p = channel_problem(B, n, k, seed=B * 7 + n + k)
    x = oconv.conv_full(p["h"], p["s"]) + p["noise"]
    r_want = oconv.conv_full(p["h_est"], p["s_est"]) - x
    wh, ws = oconv.conv_adjoint(p["s_est"], p["h_est"], r_want)
    r = torch.full((B, n + k - 1), float("nan"), device="cuda")
    gh, gs = adj.conv_gradient(dev(p["s_est"]), dev(p["h_est"]), dev(x), r=r)
    assert_close(r.cpu().numpy(), r_want, what=f"residual {B}x{n}x{k}")
    assert_close(gh.cpu().numpy(), wh, what=f"grad_h {B}x{n}x{k}")
    assert_close(gs.cpu().numpy(), ws, what=f"grad_s {B}x{n}x{k}")
    gh2, gs2 = adj.conv_gradient(dev(p["s_est"]), dev(p["h_est"]), dev(x))     # without r out
    assert torch.equal(gh2, gh) and torch.equal(gs2, gs)
    assert adj.device_status() == 0


@pytest.mark.parametrize("k", [4, 64])
def test_one_gradient_only_and_empty(adj, k):
    n = 9000
    sh, hh, rh = random_vector((2, n), 1), random_vector((2, k), 2), random_vector((2, n + k - 1), 3)
    s, h, r = dev(sh), dev(hh), dev(rh)
    wh, ws = oconv.conv_adjoint(sh, hh, rh)
    gh, gs = adj.conv_adjoint(s, h, r, grad_s=False)
    assert gs is None and gh.shape == (2, k)
    assert_close(gh.cpu().numpy(), wh, what="grad_h alone")
    gh2, gs2 = adj.conv_adjoint(s, h, r, grad_h=False)
    assert gh2 is None and gs2.shape == (2, n)
    assert_close(gs2.cpu().numpy(), ws, what="grad_s alone")
    e = torch.empty(0, n, device="cuda")
    gh, gs = adj.conv_adjoint(e, torch.empty(0, k, device="cuda"), torch.empty(0, n + k - 1, device="cuda"))
    assert gh.numel() == 0 and gs.numel() == 0


@pytest.mark.parametrize("k", [17, 64])
def test_fused_gradient_one_output(adj, k):
    """conv_gradient asked for grad_h alone or grad_s alone (the tensor-core
    kernel then skips its second product or the grad_h pass)."""
    B, n = 3, 9000
    p = channel_problem(B, n, k, seed=k + 5)
    x = oconv.conv_full(p["h"], p["s"]) + p["noise"]
    r = oconv.conv_full(p["h_est"], p["s_est"]) - x
    wh, ws = oconv.conv_adjoint(p["s_est"], p["h_est"], r)
    gh, gs = adj.conv_gradient(dev(p["s_est"]), dev(p["h_est"]), dev(x), grad_s=False)
    assert gs is None
    assert_close(gh.cpu().numpy(), wh, what=f"grad_h alone k={k}")
    gh, gs = adj.conv_gradient(dev(p["s_est"]), dev(p["h_est"]), dev(x), grad_h=False)
    assert gh is None
    assert_close(gs.cpu().numpy(), ws, what=f"grad_s alone k={k}")


@pytest.mark.parametrize("B,n,k", [(2, 8192, 61), (2, 8190, 63), (3, 8191, 62), (2, 8189, 60)])
def test_row_length_load_paths(adj, B, n, k):
    """Rows of s and of x / r are fetched 16 bytes at a time when their
    length is a multiple of 4 and 4 bytes at a time otherwise: (s, x) lengths
    (8192, 8252) both wide, (8190, 8252) and (8191, 8252) x wide only,
    (8189, 8248) x wide only as well; the residual r of conv_adjoint has the
    length of x."""
    p = channel_problem(B, n, k, seed=n + k)
    x = oconv.conv_full(p["h"], p["s"]) + p["noise"]
    r = oconv.conv_full(p["h_est"], p["s_est"]) - x
    wh, ws = oconv.conv_adjoint(p["s_est"], p["h_est"], r)
    gh, gs = adj.conv_gradient(dev(p["s_est"]), dev(p["h_est"]), dev(x))
    assert_close(gh.cpu().numpy(), wh, what=f"fused grad_h {B}x{n}x{k}")
    assert_close(gs.cpu().numpy(), ws, what=f"fused grad_s {B}x{n}x{k}")
    gh, gs = adj.conv_adjoint(dev(p["s_est"]), dev(p["h_est"]), dev(r))
    assert_close(gh.cpu().numpy(), wh, what=f"grad_h {B}x{n}x{k}")
    assert_close(gs.cpu().numpy(), ws, what=f"grad_s {B}x{n}x{k}")


def test_full_size_256x65536x64(adj):
    """The bench workload (256 signals of 65,536 samples, 64-tap channels), in full."""
    p = channel_problem(256, 65536, 64, seed=2)
    x = oconv.conv_full(p["h"], p["s"]) + p["noise"]
    r = oconv.conv_full(p["h_est"], p["s_est"]) - x
    gh, gs = adj.conv_adjoint(dev(p["s_est"]), dev(p["h_est"]), dev(r))
    wh, ws = oconv.conv_adjoint(p["s_est"], p["h_est"], r)
    assert_close(gh.cpu().numpy(), wh, what="grad_h full")
    assert_close(gs.cpu().numpy(), ws, what="grad_s full")
    gh, gs = adj.conv_gradient(dev(p["s_est"]), dev(p["h_est"]), dev(x))
    assert_close(gh.cpu().numpy(), wh, what="fused grad_h full")
    assert_close(gs.cpu().numpy(), ws, what="fused grad_s full")


@pytest.mark.parametrize("C,n,k", [(2, 1767, 844), (2, 1717, 894), (3, 300, 17), (1, 5, 3), (2, 2000, 1500)])
def test_bce_gradient_eq6(C, n, k):
    """Eq. 6 (shared source, Huber-softened TV on the channels) at the paper's
    estimated and true lengths (N_est = 1767, K_est = 844; N = 1717, K = 894),
    small cases, and k above the fused kernel's limit."""
    import paper_1707_02018_gb300 as adj
    from oracle import conv as oconv
    rng = np.random.default_rng(C * 1000 + k)
    s, H = rng.standard_normal(n), rng.standard_normal((C, k))
    X = rng.standard_normal((C, n + k - 1))
    lam_tv, delta = 0.01, 0.1  # the paper's lambda_{h,TV} and delta
    dev = lambda a: torch.as_tensor(a, dtype=torch.float32, device="cuda").contiguous()  # noqa: E731
    gh, gs = adj.bce_gradient(dev(s), dev(H), dev(X), lam_tv, delta)
    wh, ws_ = oconv.bce_gradient(s, H, X, lam_tv, delta)
    assert_close(gh.cpu().numpy(), wh, what=f"grad_h C{C} n{n} k{k}")
    assert_close(gs.cpu().numpy(), ws_, what=f"grad_s C{C} n{n} k{k}")
