"""Python binding of libadjwt (argument marshalling only).

Every operator runs in the CUDA kernels of libadjwt.so behind the C-ABI of
include/adjwt.h; this module only turns torch tensors into device pointers,
sizes and the current CUDA stream, allocates outputs and workspaces with
torch, and raises on a non-zero status.  Names follow the C-ABI.

Layouts: images are (rows, image_pitch) float32 tensors (cols rounded up to a
multiple of 4); coefficient vectors are flat (num_coeffs,) float32 tensors in
the padded packed band order of the plan.  `WtPlan.pack` / `WtPlan.unpack`
convert to and from the unpadded packed order.
"""
import ctypes as C

import torch

from . import _lib
from ._lib import AdjwtError, FistaProblem, FistaState  # noqa: F401

BC = {"zero": 0, "sym": 1, "ppd": 2, "per": 3}
WAVELET = {"haar": 0, "db2": 1, "db4": 2, "cdf97": 3}


def lib():
    return _lib.load()


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensor must live on a CUDA device")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _need(t, numel, name):
    if t.dtype != torch.float32 or not t.is_contiguous() or t.numel() < numel:
        raise ValueError(f"{name}: need a contiguous float32 CUDA tensor with >= {numel} elements")


def workspace(nbytes, device=None):
    """A 256-byte aligned scratch buffer (torch-allocated)."""
    n = max(int(nbytes), 1) + 256
    raw = torch.empty(n, dtype=torch.uint8, device=device or "cuda")
    off = (-raw.data_ptr()) % 256
    return raw[off:off + max(int(nbytes), 1)]


class WtPlan:
    """Plan of a `levels`-level 2D transform of a rows x cols image."""

    def __init__(self, rows, cols, levels, wavelet="cdf97", bc="sym"):
        self.rows, self.cols, self.levels = rows, cols, levels
        self.wavelet, self.bc = wavelet, bc
        h = C.c_void_p()
        _lib.check(lib().adjwt_wt_plan_create(C.byref(h), rows, cols, levels, WAVELET[wavelet], BC[bc]))
        self._h = h
        nb = 3 * levels + 1
        nc = C.c_int64()
        offs = (C.c_int64 * nb)()
        br, bcol, bp = (C.c_int * nb)(), (C.c_int * nb)(), (C.c_int * nb)()
        ip = C.c_int()
        _lib.check(lib().adjwt_wt_layout(h, C.byref(nc), offs, br, bcol, bp, C.byref(ip)))
        self.num_coeffs = nc.value
        self.band_offsets = list(offs)
        self.band_rows, self.band_cols, self.band_pitch = list(br), list(bcol), list(bp)
        self.image_pitch = ip.value
        self.workspace_bytes = lib().adjwt_wt_workspace_size(h)

    @property
    def handle(self):
        return self._h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib._lib is not None:
            _lib._lib.adjwt_wt_plan_destroy(h)
            self._h = None

    LEVEL_OPS = {"synth": 0, "analysis": 1, "prox": 2}

    def set_tma(self, op, level, enabled):
        """op "synth" (W), "analysis" (W^*, W^dagger) or "prox" (W^* with the
        FISTA prox epilogue): run `level` on the TMA kernel under its size rule
        (enabled) or on the tiled kernel alone."""
        _lib.check(lib().adjwt_wt_plan_set_tma(self._h, self.LEVEL_OPS[op], int(level), int(enabled)))

    def set_tma_ctas(self, op, level, ctas):
        """Cap the TMA kernel of `level` at `ctas` resident CTAs per SM (1..3; 0 = as many as fit)."""
        _lib.check(lib().adjwt_wt_plan_set_tma_ctas(self._h, self.LEVEL_OPS[op], int(level), int(ctas)))

    def tma_ctas(self):
        """{"synth", "analysis", "prox": [...]}: per level 1..J, the CTA cap of the TMA kernel (0 = none)."""
        out = {}
        for name, op in self.LEVEL_OPS.items():
            v = C.c_int()
            row = []
            for j in range(1, self.levels + 1):
                _lib.check(lib().adjwt_wt_plan_tma_ctas(self._h, op, j, C.byref(v)))
                row.append(v.value)
            out[name] = row
        return out

    def tma_levels(self):
        """{"synth", "analysis", "prox": [...]}: per level 1..J, whether the TMA kernel runs."""
        out = {}
        for name, op in self.LEVEL_OPS.items():
            v = C.c_int()
            row = []
            for j in range(1, self.levels + 1):
                _lib.check(lib().adjwt_wt_plan_uses_tma(self._h, op, j, C.byref(v)))
                row.append(bool(v.value))
            out[name] = row
        return out

    def set_level_chain(self, enabled):
        """Run the deepest tiled-only levels as one launch (True) or one launch
        per level (False, the default: measured faster on GB300)."""
        _lib.check(lib().adjwt_wt_plan_set_level_chain(self._h, int(bool(enabled))))

    def chain_start(self):
        """{"synth", "analysis", "prox": first level of the level chain, 0 = none}."""
        out = {}
        for name, op in self.LEVEL_OPS.items():
            v = C.c_int()
            _lib.check(lib().adjwt_wt_plan_chain_start(self._h, op, C.byref(v)))
            out[name] = int(v.value)
        return out

    def autotune(self, reps=5, stream=None):
        """Measure each level's implementation (tiled kernel, or TMA kernel with
        as many CTAs per SM as fit, one or two; see include/adjwt.h); True if
        the choices came from an earlier tuning of the same size class."""
        fc = C.c_int()
        _lib.check(lib().adjwt_wt_plan_autotune(self._h, int(reps), C.byref(fc), _stream(stream)))
        return bool(fc.value)

    def filters(self):
        arrs = [(C.c_double * 10)() for _ in range(4)]
        L = C.c_int()
        _lib.check(lib().adjwt_wt_filters(self._h, *arrs, C.byref(L)))
        names = ("dec_lo", "dec_hi", "rec_lo", "rec_hi")
        return {n: list(a)[:L.value] for n, a in zip(names, arrs)}

    @property
    def logical_size(self):
        return sum(r * c for r, c in zip(self.band_rows, self.band_cols))

    def pack(self, flat):
        """Unpadded packed vector (any device) -> padded device vector."""
        flat = torch.as_tensor(flat, dtype=torch.float32)
        out = torch.zeros(self.num_coeffs, dtype=torch.float32, device="cuda")
        pos = 0
        for off, r, c, p in zip(self.band_offsets, self.band_rows, self.band_cols, self.band_pitch):
            out[off:off + r * p].view(r, p)[:, :c] = flat[pos:pos + r * c].view(r, c).to(out.device)
            pos += r * c
        return out

    def unpack(self, padded):
        parts = []
        for off, r, c, p in zip(self.band_offsets, self.band_rows, self.band_cols, self.band_pitch):
            parts.append(padded[off:off + r * p].view(r, p)[:, :c].reshape(-1))
        return torch.cat(parts)

    def image(self, img=None):
        """A (rows, image_pitch) device image, zero padded, optionally filled."""
        out = torch.zeros(self.rows, self.image_pitch, dtype=torch.float32, device="cuda")
        if img is not None:
            out[:, :self.cols] = torch.as_tensor(img, dtype=torch.float32).to(out.device)
        return out


def _ws(plan_bytes, ws):
    if ws is None:
        ws = workspace(plan_bytes)
    return ws, ws.numel()


def wt_synth(plan, coeffs, image=None, ws=None, stream=None):
    """W: coefficients -> image (rows, image_pitch)."""
    _need(coeffs, plan.num_coeffs, "coeffs")
    image = plan.image() if image is None else image
    _need(image, plan.rows * plan.image_pitch, "image")
    ws, nb = _ws(plan.workspace_bytes, ws)
    _lib.check(lib().wt_synth(plan.handle, _ptr(coeffs), _ptr(image), _ptr(ws), nb, _stream(stream)))
    return image


def wt_synth_adjoint(plan, image, coeffs=None, ws=None, stream=None):
    """W^*: image (rows, image_pitch) -> coefficients."""
    _need(image, plan.rows * plan.image_pitch, "image")
    coeffs = torch.empty(plan.num_coeffs, dtype=torch.float32, device=image.device) if coeffs is None else coeffs
    _need(coeffs, plan.num_coeffs, "coeffs")
    ws, nb = _ws(plan.workspace_bytes, ws)
    _lib.check(lib().wt_synth_adjoint(plan.handle, _ptr(image), _ptr(coeffs), _ptr(ws), nb, _stream(stream)))
    return coeffs


def wt_analysis(plan, image, coeffs=None, ws=None, stream=None):
    """W^dagger: image -> coefficients (wt_synth(wt_analysis(u)) = u)."""
    _need(image, plan.rows * plan.image_pitch, "image")
    coeffs = torch.empty(plan.num_coeffs, dtype=torch.float32, device=image.device) if coeffs is None else coeffs
    _need(coeffs, plan.num_coeffs, "coeffs")
    ws, nb = _ws(plan.workspace_bytes, ws)
    _lib.check(lib().wt_analysis(plan.handle, _ptr(image), _ptr(coeffs), _ptr(ws), nb, _stream(stream)))
    return coeffs


class BlurPlan:
    """Separable PSF outer(taps_r, taps_c) under bc in {zero, sym, per}."""

    def __init__(self, rows, cols, taps_r, taps_c=None, bc="sym"):
        taps_c = taps_r if taps_c is None else taps_c
        tr = (C.c_double * len(taps_r))(*[float(v) for v in taps_r])
        tc = (C.c_double * len(taps_c))(*[float(v) for v in taps_c])
        h = C.c_void_p()
        _lib.check(lib().adjwt_blur_plan_create(C.byref(h), rows, cols, tr, len(taps_r), tc, len(taps_c), BC[bc]))
        self._h = h
        self.rows, self.cols, self.bc = rows, cols, bc
        self.image_pitch = lib().adjwt_blur_image_pitch(h)
        self.workspace_bytes = lib().adjwt_blur_workspace_size(h)

    @property
    def handle(self):
        return self._h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib._lib is not None:
            _lib._lib.adjwt_blur_plan_destroy(h)
            self._h = None

    def image(self, img=None):
        out = torch.zeros(self.rows, self.image_pitch, dtype=torch.float32, device="cuda")
        if img is not None:
            out[:, :self.cols] = torch.as_tensor(img, dtype=torch.float32).to(out.device)
        return out


def bce_gradient(s, h, x, lambda_tv, delta, ws=None, stream=None):
    """(grad_h, grad_s) of the smooth part of Eq. 6 for channels h (C, k)
    sharing the source s (n,), observations x (C, n + k - 1)."""
    C, k = h.shape
    n = s.shape[0]
    assert x.shape == (C, n + k - 1)
    gh = torch.empty(C, k, dtype=torch.float32, device=h.device)
    gs = torch.empty(n, dtype=torch.float32, device=h.device)
    wsp, nb = _ws(lib().adjwt_bce_gradient_workspace_size(C, n, k), ws)
    _lib.check(lib().bce_gradient(C, n, k, _ptr(s), _ptr(h), _ptr(x), float(lambda_tv), float(delta), _ptr(gh),
                                  _ptr(gs), _ptr(wsp), nb, _stream(stream)))
    return gh, gs


def wait_selftest(arrive, stream=None):
    """Launch the bounded-wait self-test (arrive=False: the wait runs out and
    records ADJWT_ERR_TIMEOUT in the device status word); read device_status()."""
    _lib.check(lib().adjwt_wait_selftest(int(bool(arrive)), _stream(stream)))


def device_status(clear=True):
    """Device status word (0, or ADJWT_ERR_TIMEOUT after a bounded wait gave up); synchronises."""
    v = C.c_int()
    _lib.check(lib().adjwt_device_status(C.byref(v), int(bool(clear))))
    return v.value


def blur(plan, x, out=None, stream=None):
    _need(x, plan.rows * plan.image_pitch, "in")
    out = torch.zeros_like(x) if out is None else out
    _lib.check(lib().blur(plan.handle, _ptr(x), _ptr(out), _stream(stream)))
    return out


def blur_adjoint(plan, x, out=None, stream=None):
    _need(x, plan.rows * plan.image_pitch, "in")
    out = torch.zeros_like(x) if out is None else out
    _lib.check(lib().blur_adjoint(plan.handle, _ptr(x), _ptr(out), _stream(stream)))
    return out


def blur_normal(plan, u, b=None, g=None, want_norm=False, ws=None, stream=None, scratch=True):
    """g = R^*(R u - b); with want_norm also returns 1/2 ||R u - b||^2 (float64 device scalar).

    With a workspace (scratch=True or want_norm) radii <= 12 run as two
    TMA-staged passes through a scratch image; without one, as a single
    fused tiled kernel."""
    _need(u, plan.rows * plan.image_pitch, "u")
    g = torch.zeros_like(u) if g is None else g
    half = None
    wsp, nb = (None, 0)
    if want_norm:
        half = torch.zeros(1, dtype=torch.float64, device=u.device)
    if want_norm or scratch or ws is not None:
        wsp, nb = _ws(plan.workspace_bytes, ws)
    _lib.check(lib().blur_normal(plan.handle, _ptr(u), _ptr(b), _ptr(g), _ptr(half), _ptr(wsp), nb, _stream(stream)))
    return (g, half) if want_norm else g


def conv_adjoint(s, h, r, grad_h=True, grad_s=True, ws=None, stream=None):
    """(grad_h, grad_s) of Eq. 5 for batched rows s (B, n), h (B, k), r (B, n+k-1)."""
    B, n = s.shape
    k = h.shape[1]
    assert r.shape == (B, n + k - 1)
    gh = torch.empty(B, k, dtype=torch.float32, device=r.device) if grad_h is True else grad_h
    gs = torch.empty(B, n, dtype=torch.float32, device=r.device) if grad_s is True else grad_s
    gh = None if gh is False else gh
    gs = None if gs is False else gs
    nbytes = lib().adjwt_conv_adjoint_workspace_size(B, n, k)
    wsp, nb = _ws(nbytes, ws)
    _lib.check(lib().conv_adjoint(B, n, k, _ptr(s), _ptr(h), _ptr(r), _ptr(gh), _ptr(gs), _ptr(wsp), nb,
                                  _stream(stream)))
    return gh, gs


def conv_gradient(s, h, x=None, r=None, grad_h=True, grad_s=True, ws=None, stream=None):
    """(grad_h, grad_s) of Eq. 5 at (h, s) with r = h * s - x formed in the same pass.
    Pass a (B, n+k-1) tensor as r to also receive the residual."""
    B, n = s.shape
    k = h.shape[1]
    gh = torch.empty(B, k, dtype=torch.float32, device=s.device) if grad_h is True else grad_h
    gs = torch.empty(B, n, dtype=torch.float32, device=s.device) if grad_s is True else grad_s
    gh = None if gh is False else gh
    gs = None if gs is False else gs
    nbytes = lib().adjwt_conv_gradient_workspace_size(B, n, k)
    wsp, nb = _ws(nbytes, ws)
    _lib.check(lib().conv_gradient(B, n, k, _ptr(s), _ptr(h), _ptr(x), _ptr(r), _ptr(gh), _ptr(gs), _ptr(wsp), nb,
                                   _stream(stream)))
    return gh, gs


def conv_residual(h, s, x=None, r=None, stream=None):
    B, n = s.shape
    k = h.shape[1]
    r = torch.empty(B, n + k - 1, dtype=torch.float32, device=s.device) if r is None else r
    _lib.check(lib().conv_residual(B, n, k, _ptr(h), _ptr(s), _ptr(x), _ptr(r), _stream(stream)))
    return r


class Fista:
    """FISTA state and problem for min 1/2||R W x - b||^2 + lam ||x||_1 on one GPU."""

    GRADIENT = {"adjoint": 0, "pinv": 1}

    def __init__(self, wt_plan, blur_plan, b, lam, lipschitz=1.0, gradient="adjoint"):
        """gradient="pinv" puts W^dagger where W^* belongs (the comparison the paper makes)."""
        self.wt, self.blur, self.b = wt_plan, blur_plan, b
        self.problem = FistaProblem(wt_plan.handle, blur_plan.handle, b.data_ptr(), float(lam), float(lipschitz),
                                    self.GRADIENT[gradient])
        self.ws = workspace(lib().adjwt_fista_workspace_size(C.byref(self.problem)))
        self.x = torch.zeros(wt_plan.num_coeffs, dtype=torch.float32, device="cuda")
        self.y = torch.zeros_like(self.x)
        self.state = FistaState(self.x.data_ptr(), self.y.data_ptr(), 1.0, 0)

    def set_lipschitz(self, L):
        self.problem.lipschitz = float(L)

    def set_observation(self, b):
        """Point the problem at another observation image b (same plan layout);
        later calls read it, so a caller can double-buffer its input copies."""
        if tuple(b.shape) != tuple(self.b.shape) or b.dtype != self.b.dtype or not b.is_cuda:
            raise ValueError("set_observation: b must match the plan's image layout")
        self.b = b
        self.problem.b = b.data_ptr()

    def reset(self, x0=None):
        self.x.zero_()
        if x0 is not None:
            self.x.copy_(x0)
        self.y.copy_(self.x)
        self.state.t = 1.0
        self.state.k = 0

    def step(self, objective=False, stream=None):
        out = C.c_double()
        _lib.check(lib().fista_step(C.byref(self.problem), C.byref(self.state), _ptr(self.ws), self.ws.numel(),
                                    C.byref(out) if objective else None, _stream(stream)))
        return out.value if objective else None

    def reset_device(self, x0=None, stream=None):
        """Start a solve whose momentum lives on the device: x = y = x0 (or 0), t = 1."""
        st = stream if stream is not None else torch.cuda.current_stream()
        with torch.cuda.stream(st):
            self.x.zero_()
            if x0 is not None:
                self.x.copy_(x0)
            self.y.copy_(self.x)
        _lib.check(lib().adjwt_fista_device_reset(C.byref(self.problem), _ptr(self.ws), self.ws.numel(), _stream(st)))

    def step_device(self, objective_out=None, stream=None):
        """One iteration with no host state and no synchronisation (capturable
        in a CUDA graph); objective_out: optional 1-element float64 device
        tensor that receives F(x_k)."""
        _lib.check(lib().fista_step_device(C.byref(self.problem), _ptr(self.x), _ptr(self.y), _ptr(self.ws),
                                           self.ws.numel(), _ptr(objective_out), _stream(stream)))

    def objective(self, x=None, stream=None):
        out = C.c_double()
        x = self.x if x is None else x
        _lib.check(lib().adjwt_fista_objective(C.byref(self.problem), _ptr(x), _ptr(self.ws), self.ws.numel(),
                                               C.byref(out), _stream(stream)))
        return out.value

    def vjp_workspace(self):
        """Scratch for fista_vjp_step on this problem."""
        return workspace(lib().adjwt_fista_vjp_workspace_size(C.byref(self.problem)), device=self.x.device)

    def lipschitz(self, v, iters=50, stream=None):
        out = C.c_double()
        _lib.check(lib().adjwt_fista_lipschitz(C.byref(self.problem), _ptr(v), iters, _ptr(self.ws),
                                               self.ws.numel(), C.byref(out), _stream(stream)))
        return out.value


# ------------------------------------------------------------ differentiation
class FistaBatch:
    """Many FISTA problems advanced together by the batched engine (one
    persistent launch per call of run(); see include/adjwt.h).  `fistas`: Fista
    objects whose problem (plans, b, lambda, L_f, gradient) and state buffers
    (x, y) the batch uses; they must outlive it."""

    def __init__(self, fistas):
        self.fistas = list(fistas)
        n = len(self.fistas)
        self._probs = (FistaProblem * n)(*[f.problem for f in self.fistas])
        self._x = (C.c_void_p * n)(*[f.x.data_ptr() for f in self.fistas])
        self._y = (C.c_void_p * n)(*[f.y.data_ptr() for f in self.fistas])
        nbytes = lib().adjwt_fista_batch_workspace_size(n, self._probs)
        if nbytes == 0:
            raise ValueError("FistaBatch: invalid problems")
        self.ws = workspace(nbytes)
        h = C.c_void_p()
        _lib.check(lib().adjwt_fista_batch_create(C.byref(h), n, self._probs, self._x, self._y, _ptr(self.ws),
                                                  self.ws.numel()))
        self._h = h
        self.objectives = torch.zeros(n, dtype=torch.float64, device="cuda")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib._lib is not None:
            _lib._lib.adjwt_fista_batch_destroy(h)
            self._h = None

    def reset(self, stream=None):
        """x = y = 0 and t = 1 for every problem."""
        st = stream if stream is not None else torch.cuda.current_stream()
        with torch.cuda.stream(st):
            for f in self.fistas:
                f.x.zero_()
                f.y.zero_()
        _lib.check(lib().adjwt_fista_batch_reset(self._h, _stream(stream)))

    def set_momentum(self, k, stream=None):
        """Momentum of every problem as after k iterations from t_1 = 1 (x and
        y untouched): continues runs that a rebuilt batch takes over."""
        _lib.check(lib().adjwt_fista_batch_set_iteration(self._h, int(k), _stream(stream)))

    def run(self, iters, stream=None):
        _lib.check(lib().adjwt_fista_batch_run(self._h, int(iters), _stream(stream)))

    def objective(self, stream=None):
        """F(x_i) of every problem into self.objectives (device float64)."""
        _lib.check(lib().adjwt_fista_batch_objective(self._h, _ptr(self.objectives), _stream(stream)))
        return self.objectives

    def wait_selftest(self, stream=None):
        _lib.check(lib().adjwt_fista_batch_wait_selftest(self._h, _stream(stream)))

    def info(self):
        items, stages, ctas = C.c_int(), C.c_int(), C.c_int()
        _lib.check(lib().adjwt_fista_batch_info(self._h, C.byref(items), C.byref(stages), C.byref(ctas)))
        return {"items_per_iteration": items.value, "stages": stages.value, "ctas": ctas.value}


def fista_momentum(t):
    """(beta_k, t_{k+1}) of FISTA's momentum as fista_step applies it; beta_k is
    the float32 weight of y_{k+1} = x_k + beta_k (x_k - x_{k-1})."""
    t1, beta = C.c_double(), C.c_float()
    _lib.check(lib().adjwt_fista_momentum(float(t), C.byref(t1), C.byref(beta)))
    return float(beta.value), float(t1.value)


def gaussian_taps(k, sigma):
    """(taps, d taps / d sigma) of the normalised k-tap Gaussian (host lists)."""
    taps, dt = (C.c_double * k)(), (C.c_double * k)()
    _lib.check(lib().adjwt_gaussian_taps(int(k), float(sigma), taps, dt))
    return list(taps), list(dt)


def axpby(a, x, b, y, out=None, stream=None):
    """out = a x + b y (float32 device tensors of one length)."""
    if x.numel() != y.numel():
        raise ValueError("axpby: x and y differ in length")
    out = torch.empty_like(x) if out is None else out
    _need(out, x.numel(), "out")
    _lib.check(lib().adjwt_axpby(x.numel(), float(a), _ptr(x), float(b), _ptr(y), _ptr(out), _stream(stream)))
    return out


def soft_threshold(x, tau, out=None, stream=None):
    """out = sign(x) max(|x| - tau, 0) (the FISTA prox's soft threshold)."""
    out = torch.empty_like(x) if out is None else out
    _need(out, x.numel(), "out")
    _lib.check(lib().adjwt_soft_threshold(x.numel(), _ptr(x), float(tau), _ptr(out), _stream(stream)))
    return out


_reduce_ws = {}


def _reduce_scratch(device):
    key = torch.device(device).index
    if key not in _reduce_ws:
        _reduce_ws[key] = workspace(lib().adjwt_reduce_workspace_size(), device=device)
    return _reduce_ws[key]


def dot(x, y, rows=1, cols=None, pitch=None, out=None, stream=None):
    """<x, y> in float64 into a 1-element device tensor: x and y hold `rows`
    rows of `cols` values at row pitch `pitch` (default: one flat vector)."""
    cols = x.numel() if cols is None else cols
    pitch = cols if pitch is None else pitch
    _need(x, rows * pitch, "x")
    _need(y, rows * pitch, "y")
    out = torch.zeros(1, dtype=torch.float64, device=x.device) if out is None else out
    ws = _reduce_scratch(x.device)
    _lib.check(lib().adjwt_dot(rows, cols, pitch, _ptr(x), _ptr(y), _ptr(out), _ptr(ws), ws.numel(),
                               _stream(stream)))
    return out


def prox_vjp(x_next, xbar, zbar=None, stream=None):
    """(zbar, s): zbar = xbar where x_next != 0 else 0, s (1-element float64
    device tensor) = sum sign(x_next) xbar; d loss / d tau = -s."""
    zbar = torch.empty_like(xbar) if zbar is None else zbar
    s = torch.zeros(1, dtype=torch.float64, device=xbar.device)
    ws = _reduce_scratch(xbar.device)
    _lib.check(lib().fista_prox_vjp(x_next.numel(), _ptr(x_next), _ptr(xbar), _ptr(zbar), _ptr(s), _ptr(ws),
                                    ws.numel(), _stream(stream)))
    return zbar, s


def fista_vjp_step(fista, dblur, x_next, y_k, beta, xbar, ybar, db, dtau, dsigma, ws, stream=None):
    """One reverse-mode step of FISTA iteration k in a single library call:
    xbar (adjoint of x_{k+1}) and ybar (adjoint of y_{k+1}) are replaced by
    the adjoints of x_k (from y_{k+1}) and y_k, db (image or None) gains
    (1/L) R W zbar, and the float64 device scalars dtau / dsigma accumulate
    dl/dtau and dl/dsigma.  dblur: the two plans of dR/dsigma, or None with
    dsigma None.  ws: fista.vjp_workspace()."""
    d1, d2 = (None, None) if dblur is None else (dblur[0].handle, dblur[1].handle)
    _lib.check(lib().fista_vjp_step(C.byref(fista.problem), d1, d2, _ptr(x_next), _ptr(y_k), float(beta), _ptr(xbar),
                                    _ptr(ybar), None if db is None else _ptr(db), _ptr(dtau),
                                    None if dsigma is None else _ptr(dsigma), _ptr(ws), ws.numel(), _stream(stream)))


def fista_step(fista, objective=False, stream=None):
    return fista.step(objective, stream)


def trace_enable(capacity):
    """Arm (capacity > 0) or disarm (0) per-kernel event timing in libadjwt."""
    _lib.check(lib().adjwt_trace_enable(int(capacity)))


def trace_level(level):
    """1: time every kernel (default); 2: time whole operator calls only ("op:..." records)."""
    _lib.check(lib().adjwt_trace_set_level(int(level)))


def trace_reset():
    _lib.check(lib().adjwt_trace_reset())


def fp32_fma_peak(stream=None):
    """Measured float32 FMA rate of the current device, TFLOP/s."""
    v = C.c_double()
    _lib.check(lib().adjwt_fp32_fma_peak(C.byref(v), _stream(stream)))
    return float(v.value)


def trace_span(first, last):
    """Device milliseconds from the start of trace record `first` to the end of `last`."""
    ms = C.c_float()
    _lib.check(lib().adjwt_trace_span(int(first), int(last), C.byref(ms)))
    return float(ms.value)


def trace_records():
    """[(kernel name, tag, milliseconds)] of the armed trace (waits for each record)."""
    out = []
    name, tag, ms = C.c_char_p(), C.c_int(), C.c_float()
    for i in range(lib().adjwt_trace_count()):
        _lib.check(lib().adjwt_trace_get(i, C.byref(name), C.byref(tag), C.byref(ms)))
        out.append((name.value.decode(), tag.value, ms.value))
    return out
