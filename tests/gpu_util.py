"""Shared helpers of the GPU parity tests (tolerance checks, layout moves)."""
import numpy as np
import torch

# Per-operator tolerance: ||gpu - oracle||_2 / ||oracle||_2 <= 1e-5 (float32
# kernels against the float64 oracle); the elementwise bound scales with the
# largest oracle magnitude because relative error is undefined at zeros.
REL_L2 = 1e-5
ABS_MAX = 2e-5


def rel_err(got, want):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    den = np.linalg.norm(want)
    num = np.linalg.norm(got - want)
    return num / den if den > 0 else num


def assert_close(got, want, rel=REL_L2, abs_max=ABS_MAX, what=""):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    assert got.shape == want.shape, (what, got.shape, want.shape)
    assert np.all(np.isfinite(got)), what
    r = rel_err(got, want)
    scale = max(np.abs(want).max(), 1e-30)
    m = np.abs(got - want).max() / scale
    assert r <= rel and m <= abs_max, f"{what}: rel L2 {r:.3e} (<= {rel}), max abs / scale {m:.3e} (<= {abs_max})"
    return r, m


def to_host_image(t, rows, cols):
    return t[:, :cols].double().cpu().numpy()


def image_dev(plan, img):
    return plan.image(torch.as_tensor(np.asarray(img), dtype=torch.float32))
