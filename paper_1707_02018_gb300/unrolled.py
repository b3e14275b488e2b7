"""Unrolled FISTA on the GPU and its reverse mode (gradients with respect to
lambda, the Gaussian PSF width sigma and the observation b).

The solve of Eq. 1, min_x 1/2 ||R W x - b||^2 + lambda ||x||_1, run for N
FISTA iterations from x_0 = y_0 = 0 with a constant step 1/L, is a
differentiable map of (lambda, sigma, b) almost everywhere.  Its backward
applies A = R W and A^* = W^* R^* (the chain rule of Sec. I: the gradient of
l(A x) is A^* grad l, right only with the exact adjoint W^* of Eq. 4) and
dR/dsigma = R[g', g] + R[g, g'] for the separable Gaussian g (x) g.  With
beta_k = (t_k - 1)/t_{k+1} the momentum factor of iteration k and the loss
l = 1/2 ||W x_N - u_ref||^2, going back from k = N-1 to 0 (Xp: adjoint of
x_{k+1} collected so far, Y: adjoint of y_{k+1}):
    X     = Xp + (1 + beta_k) Y
    zbar  = X where x_{k+1} != 0;   dl/dtau -= sum sign(x_{k+1}) X
    u     = W zbar
    Y_k   = zbar - (1/L) W^* R^* R u;   Xp = -beta_k Y;   dl/db += (1/L) R u
    dl/dsigma -= (1/L) (<R' u, R W y_k - b> + <R u, R' W y_k>)
and dl/dlambda = dl/dtau / L.  L is held fixed.  Every vector step is one of
the library's kernels (W, W^*, R, R^*, the soft-threshold VJP, a x + b y,
float64 inner products); by default one backward iteration is one library
call (fista_vjp_step) that issues them all, with dl/dtau and dl/dsigma
accumulated on the device.  The iterates are kept at checkpoints only and the
segments between them recomputed during the backward pass.
"""
import math

import torch

from . import (BlurPlan, Fista, WtPlan, axpby, blur, blur_adjoint, dot, fista_momentum, fista_vjp_step,
               gaussian_taps, prox_vjp, wt_synth, wt_synth_adjoint)


class UnrolledFista:
    """N-step FISTA for one problem; `grads` returns (loss, dl/dlam, dl/dsigma, dl/db)."""

    def __init__(self, rows, cols, levels, wavelet, mode, k, sigma, blur_bc, b, lam, L):
        g, dg = gaussian_taps(k, sigma)
        self.wt = WtPlan(rows, cols, levels, wavelet, mode)
        self.R = BlurPlan(rows, cols, g, g, blur_bc)
        self.dR = (BlurPlan(rows, cols, dg, g, blur_bc), BlurPlan(rows, cols, g, dg, blur_bc))
        if self.R.image_pitch != self.wt.image_pitch:
            raise ValueError("wavelet and blur plans disagree on the image pitch")
        self.rows, self.cols, self.pitch = rows, cols, self.wt.image_pitch
        self.b = b
        self.lam, self.L = float(lam), float(L)
        self.fista = Fista(self.wt, self.R, b, self.lam, self.L)
        self._vjp_ws = None

    # --------------------------------------------------------------- helpers
    def _img_dot(self, x, y):
        return dot(x, y, rows=self.rows, cols=self.cols, pitch=self.pitch)

    def _dR(self, u):
        return axpby(1.0, blur(self.dR[0], u), 1.0, blur(self.dR[1], u))

    def _run(self, start, stop, keep):
        """Iterations start .. stop-1 from the state already in self.fista;
        returns the iterates (x_k, y_k) for k in start .. stop if keep."""
        f = self.fista
        xs, ys = ([f.x.clone()], [f.y.clone()]) if keep else (None, None)
        for _ in range(start, stop):
            f.step()
            if keep:
                xs.append(f.x.clone())
                ys.append(f.y.clone())
        return xs, ys

    # ----------------------------------------------------------------- public
    def solve(self, n_steps):
        """x_N after n_steps iterations from zero."""
        self.fista.reset()
        self._run(0, n_steps, keep=False)
        return self.fista.x.clone()

    def _back_pieces(self, k, beta, x_next, y_k, Xp, Y, db, tau_terms, sigma_terms):
        """Backward iteration k from the library's separate pieces; returns (Xp, Y)."""
        inv_l = 1.0 / self.L
        X = axpby(1.0, Xp, 1.0 + beta, Y)
        zbar, sd = prox_vjp(x_next, X)
        tau_terms.append(sd)
        u = wt_synth(self.wt, zbar)
        Ru = blur(self.R, u)
        q = wt_synth_adjoint(self.wt, blur_adjoint(self.R, Ru))
        Y_k = axpby(1.0, zbar, -inv_l, q)
        Xp = axpby(-beta, Y, 0.0, Y)
        axpby(1.0, db, inv_l, Ru, out=db)
        Wy = wt_synth(self.wt, y_k)
        r = axpby(1.0, blur(self.R, Wy), -1.0, self.b)
        sigma_terms.append(-inv_l * self._img_dot(self._dR(u), r))
        sigma_terms.append(-inv_l * self._img_dot(Ru, self._dR(Wy)))
        return Xp, Y_k

    def grads(self, n_steps, u_ref, checkpoint_every=None, fused=True):
        """(loss, dl/dlambda, dl/dsigma, dl/db) for l = 1/2 ||W x_N - u_ref||^2;
        u_ref and the returned dl/db are (rows, image_pitch) device images.
        fused=False runs each backward iteration as separate library calls."""
        every = checkpoint_every or max(1, int(math.isqrt(n_steps)))
        f = self.fista
        f.reset()
        ckpt, betas = {}, []
        t = 1.0
        for k in range(n_steps):
            if k % every == 0:
                ckpt[k] = (f.x.clone(), f.y.clone(), t)
            beta, t1 = fista_momentum(t)
            betas.append(beta)
            f.step()
            t = t1
        xN = f.x.clone()

        e = axpby(1.0, wt_synth(self.wt, xN), -1.0, u_ref)
        loss = 0.5 * float(self._img_dot(e, e))
        Xp = wt_synth_adjoint(self.wt, e)
        Y = torch.zeros_like(Xp)
        db = torch.zeros_like(self.b)
        dev = Xp.device
        acc = torch.zeros(2, dtype=torch.float64, device=dev)  # dl/dtau, dl/dsigma
        tau_terms, sigma_terms = [acc[0:1]], [acc[1:2]]
        if fused and self._vjp_ws is None:
            self._vjp_ws = f.vjp_workspace()
        inv_l = 1.0 / self.L
        for s in sorted(ckpt, reverse=True):
            stop = min(s + every, n_steps)
            x0, y0, t0 = ckpt[s]
            f.x.copy_(x0)
            f.y.copy_(y0)
            f.state.t, f.state.k = t0, s
            xs, ys = self._run(s, stop, keep=True)  # xs[i] = x_{s+i}
            for k in range(stop - 1, s - 1, -1):
                if fused:
                    fista_vjp_step(f, self.dR, xs[k + 1 - s], ys[k - s], betas[k], Xp, Y, db, acc[0:1], acc[1:2],
                                   self._vjp_ws)
                else:
                    Xp, Y = self._back_pieces(k, betas[k], xs[k + 1 - s], ys[k - s], Xp, Y, db, tau_terms,
                                              sigma_terms)
        dtau = -sum(float(v) for v in tau_terms[1:]) + float(acc[0])
        dsigma = sum(float(v) for v in sigma_terms)
        return loss, dtau * inv_l, dsigma, db


class UnrolledFistaLoss(torch.autograd.Function):
    """loss = 1/2 ||W x_N(lam, sigma, b) - u_ref||^2 as an autograd node whose
    backward is the reverse mode above (lam and sigma: 0-d float64 tensors;
    b: the (rows, image_pitch) observation image)."""

    @staticmethod
    def forward(ctx, lam, sigma, b, u_ref, spec, n_steps, L, checkpoint_every=None):
        rows, cols, levels, wavelet, mode, k, blur_bc = spec
        un = UnrolledFista(rows, cols, levels, wavelet, mode, k, float(sigma), blur_bc, b.detach().contiguous(),
                           float(lam), L)
        loss, dlam, dsig, db = un.grads(n_steps, u_ref.contiguous(), checkpoint_every)
        ctx.save_for_backward(db)
        ctx.dlam, ctx.dsig = dlam, dsig
        return torch.tensor(loss, dtype=torch.float64)

    @staticmethod
    def backward(ctx, g):
        (db,) = ctx.saved_tensors
        gv = float(g)
        return (torch.tensor(gv * ctx.dlam, dtype=torch.float64), torch.tensor(gv * ctx.dsig, dtype=torch.float64),
                axpby(gv, db, 0.0, db), None, None, None, None, None)


def unrolled_loss(lam, sigma, b, u_ref, spec, n_steps, L, checkpoint_every=None):
    return UnrolledFistaLoss.apply(lam, sigma, b, u_ref, spec, n_steps, L, checkpoint_every)


def _main():
    """Gradient of the unrolled loss for seeded problems
    (python -m paper_1707_02018_gb300.unrolled --batch 4 --size 512 --steps 10):
    piecewise-smooth images u, observations b = R u + noise (9 x 9 Gaussian,
    sigma 1.5, symmetric boundary), 4-level db4 with symmetric boundaries,
    lambda = 1e-3.  Prints the losses and the seconds of forward and gradient."""
    import argparse
    import time

    from synthetic_inputs import gaussian_noise, piecewise_smooth_image, random_vector

    ap = argparse.ArgumentParser()
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--steps", type=int, default=10)
    args = ap.parse_args()
    size, k, sigma, lam = args.size, 9, 1.5, 1e-3
    g, _ = gaussian_taps(k, sigma)
    runs = []
    for i in range(args.batch):
        wt = WtPlan(size, size, 4, "db4", "sym")
        bl = BlurPlan(size, size, g, g, "sym")
        img = wt.image(torch.as_tensor(piecewise_smooth_image(size, size, 900 + i)))
        b = blur(bl, img)
        b[:, :size] += torch.as_tensor(gaussian_noise((size, size), 950 + i, 1e-3), dtype=torch.float32,
                                       device="cuda")
        L = Fista(wt, bl, b, lam, 1.0).lipschitz(wt.pack(random_vector(wt.logical_size, 990 + i)), iters=30)
        runs.append((UnrolledFista(size, size, 4, "db4", "sym", k, sigma, "sym", b, lam, L), img))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = [un.grads(args.steps, img) for un, img in runs]
    torch.cuda.synchronize()
    print("losses", " ".join(f"{o[0]:.4e}" for o in out), f"gradient_sec {time.perf_counter() - t0:.4f}")


if __name__ == "__main__":
    _main()
