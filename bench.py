"""Throughput of the adjoint-wavelet FISTA gradient path on GB300.

One step = one pass of the whole hot path over the 2048 x 2048 workload:
  * one FISTA iteration (W, fused R^*(R W y - b), W^* with the prox epilogue)
    for each of three deblurring problems: 5-level CDF 9/7 with periodic,
    half-point symmetric and zero boundaries, 15 x 15 Gaussian PSF (sigma 3)
    under the same boundary;
  * the blind-channel gradient of a batch of 256 signals of 65,536 samples with
    64-tap channels: residual r = h * s - x, then grad_h and grad_s.
value = algorithmic HBM bytes of the step (each operator reads its inputs and
writes its outputs once) / device time, summed over ranks, in GB/s.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs its own independent copy of the workload (weak
scaling, no data-path collective).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SIZE, LEVELS, WAVELET = 2048, 5, "cdf97"
PSF_K, PSF_SIGMA, LAM, NOISE = 15, 3.0, 1e-3, 1e-3
BCS = ("per", "sym", "zero")
# bench.py --autotune measures the TMA / tiled choice per wavelet level first
# (adjwt_wt_plan_autotune, each transform timed alone).  Off by default: the
# serially measured choice (tiled kernels for the level-1 W^* + prox) cuts the
# serial kernel time but makes this four-stream step slower.
AUTOTUNE = False
CH_B, CH_N, CH_K = 256, 65536, 64
METRIC = "W/W* HBM GB/s; FISTA sec to 1e-4 rel objective, learned/batched vs plain"
WORKLOAD = ("FISTA iteration on 2048x2048, 5-level CDF 9/7, PER+SYM+ZERO boundaries, 15x15 Gaussian PSF "
            "sigma=3, lambda=1e-3 (one problem per boundary) + blind-channel gradient 256 x 65536 samples, "
            "64-tap channels (residual + grad_h + grad_s)")


def gaussian_taps(k, sigma):
    c = (k - 1) / 2.0
    t = np.exp(-((np.arange(k) - c) ** 2) / (2.0 * sigma * sigma))
    return t / t.sum()


def level_sizes(n, levels, bc, L=10):
    out = []
    for _ in range(levels):
        m = n // 2 if bc == "per" else (n + 3 * (L - 1)) // 2
        out.append((n, m))
        n = m
    return out


def fista_bytes(bc):
    """Algorithmic float32 bytes of one fused FISTA iteration (per kernel family)."""
    lv = level_sizes(SIZE, LEVELS, bc)
    N2 = SIZE * SIZE
    C = sum(3 * m * m for _, m in lv) + lv[-1][1] ** 2
    I = sum(m * m for _, m in lv[:-1])
    return {"wt_synth": 4 * (C + N2 + 2 * I), "blur_normal": 4 * 3 * N2,
            "wt_adjoint_prox": 4 * (4 * C + N2 + 2 * I), "total": 4 * (5 * C + 5 * N2 + 4 * I),
            "level1": {"wt_synth": 4 * (4 * lv[0][1] ** 2 + N2),
                       "wt_adjoint_prox": 4 * (N2 + 13 * lv[0][1] ** 2)}}


def channel_bytes():
    """Fused channel gradient: reads s, h, x; writes grad_s, grad_h (r stays on chip)."""
    B, n, k = CH_B, CH_N, CH_K
    total = 4 * (B * n + B * k + B * (n + k - 1) + B * n + B * k)
    return {"conv_gradient": total, "total": total,
            "flops": 2 * B * (n + k - 1) * k + 4 * B * n * k}


# DRAM bytes (read + write) of one launch of the bench workload, measured by ncu on the current kernels
# (an entry is removed whenever its kernel changes, until it is captured again)
NCU_TRAFFIC = {"conv_gradient": 134448896 + 35901440,
               # k_conv32_tc<false>, 8 x 512^2 (one ncu capture: dram read + write bytes per launch)
               "cnn_conv32_tc": 134286848 + 84610304}


def step_bytes():
    return sum(fista_bytes(bc)["total"] for bc in BCS) + channel_bytes()["total"]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d["hbm_gbs"], "sm_max_mhz": d.get("sm_max_mhz", 2070.0), "source": "measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.path = index, None, None

    def start(self):
        try:
            import tempfile
            self.path = tempfile.mktemp(suffix=".csv")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        rows = [ln.split(",") for ln in open(self.path).read().strip().splitlines() if ln.strip()]
        os.unlink(self.path)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ our arm
def build_workload(adj, torch, rank):
    from synthetic_inputs import channel_problem, gaussian_noise, piecewise_smooth_image, random_vector
    p = gaussian_taps(PSF_K, PSF_SIGMA)
    probs = []
    for i, bc in enumerate(BCS):
        seed = 2000 + 10 * rank + i
        wt = adj.WtPlan(SIZE, SIZE, LEVELS, WAVELET, bc)
        if AUTOTUNE:
            wt.autotune(reps=5)  # plan-time choice of TMA / tiled kernels per level (untimed setup)
        bl = adj.BlurPlan(SIZE, SIZE, p, p, bc)
        img = wt.image(torch.as_tensor(piecewise_smooth_image(SIZE, SIZE, seed)))
        b = adj.blur(bl, img)
        b[:, :SIZE] += torch.as_tensor(gaussian_noise((SIZE, SIZE), seed + 1, NOISE), dtype=torch.float32,
                                       device="cuda")
        f = adj.Fista(wt, bl, b, LAM, 1.0)
        v0 = wt.pack(random_vector(wt.logical_size, seed + 2))
        f.set_lipschitz(f.lipschitz(v0, iters=30))
        probs.append({"bc": bc, "wt": wt, "bl": bl, "b": b, "fista": f, "b_host": b.cpu().pin_memory()})
    cp = channel_problem(CH_B, CH_N, CH_K, seed=3000 + rank)
    dev = lambda a: torch.as_tensor(a, dtype=torch.float32, device="cuda").contiguous()  # noqa: E731
    h, s = dev(cp["h"]), dev(cp["s"])
    x = adj.conv_residual(h, s) + dev(cp["noise"])
    ch = {"s": dev(cp["s_est"]), "h": dev(cp["h_est"]), "x": x,
          "gh": torch.empty(CH_B, CH_K, device="cuda"), "gs": torch.empty(CH_B, CH_N, device="cuda")}
    ch["ws"] = adj.workspace(adj.lib().adjwt_conv_gradient_workspace_size(CH_B, CH_N, CH_K))
    for key in ("s", "h", "x"):
        ch[key + "_host"] = ch[key].cpu().pin_memory()
    return probs, ch


class Lanes:
    """One CUDA stream per independent problem (the three boundary problems and
    the channel gradient), forked from and joined back into the caller's stream.
    The FISTA lanes get the high stream priority: their level kernels are short
    and latency bound, so the block scheduler gives them SMs first and the
    throughput-bound channel gradient (last lane) fills the rest."""

    def __init__(self, torch, n):
        self.torch = torch
        lo, hi = torch.cuda.Stream.priority_range() if hasattr(torch.cuda.Stream, "priority_range") else (0, -1)
        self.streams = [torch.cuda.Stream(priority=hi) for _ in range(n - 1)] + [torch.cuda.Stream(priority=lo)]
        self.events = [torch.cuda.Event() for _ in range(n + 1)]

    def fork(self):
        main = self.torch.cuda.current_stream()
        self.events[-1].record(main)
        for st in self.streams:
            st.wait_event(self.events[-1])

    def join(self):
        main = self.torch.cuda.current_stream()
        for ev, st in zip(self.events, self.streams):
            ev.record(st)
            main.wait_event(ev)


def max_over_ranks(torch, dist, ms, world, device):
    """The slowest rank's time (every rank gets it): ranks run independent
    replicas, so the whole job is done when the last one is."""
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(bytes_per_step, steps, world, ms):
    """GB/s of the whole job: every rank processed `steps` steps of
    `bytes_per_step` algorithmic bytes in at most `ms` milliseconds."""
    return bytes_per_step * steps * world / (ms * 1e-3) / 1e9


def pinned_h2d_rate(torch, nbytes=512 << 20, reps=5):
    """One large host -> device copy from pinned memory (the bound of the e2e
    figure), best of `reps`, CUDA events on the copying stream."""
    src = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    dst = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = torch.cuda.Stream()
    best = None
    with torch.cuda.stream(st):
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            dst.copy_(src, non_blocking=True)
            e1.record(st)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
    del src, dst
    return {"gbs": nbytes / (best * 1e-3) / 1e9, "bytes": nbytes, "how": "one pinned host -> device copy, best of 5"}


def run_step(adj, probs, ch, lanes=None):
    """One step.  With `lanes` the four independent problems run on their own
    streams (the GPU overlaps them); without, one after the other on the
    current stream."""
    if lanes is None:
        for pr in probs:
            pr["fista"].step()
        adj.conv_gradient(ch["s"], ch["h"], ch["x"], grad_h=ch["gh"], grad_s=ch["gs"], ws=ch["ws"])
        return
    lanes.fork()
    for pr, st in zip(probs, lanes.streams):
        pr["fista"].step(stream=st)
    adj.conv_gradient(ch["s"], ch["h"], ch["x"], grad_h=ch["gh"], grad_s=ch["gs"], ws=ch["ws"],
                      stream=lanes.streams[-1])
    lanes.join()


def run_step_device(adj, probs, ch, lanes=None):
    """The step with the momentum on the device (fista_step_device): the
    stream sequence that is captured in the CUDA graph the timed loop
    replays.  Without `lanes`, serially on the current stream."""
    if lanes is None:
        for pr in probs:
            pr["fista"].step_device()
        adj.conv_gradient(ch["s"], ch["h"], ch["x"], grad_h=ch["gh"], grad_s=ch["gs"], ws=ch["ws"])
        return
    lanes.fork()
    for pr, st in zip(probs, lanes.streams):
        pr["fista"].step_device(stream=st)
    adj.conv_gradient(ch["s"], ch["h"], ch["x"], grad_h=ch["gh"], grad_s=ch["gs"], ws=ch["ws"],
                      stream=lanes.streams[-1])
    lanes.join()


def capture_step(adj, torch, probs, ch, lanes):
    """One step (three FISTA iterations on their streams + the channel
    gradient) captured in a CUDA graph: every replay runs all of its kernels
    again (the iterations advance; t_k lives in each problem's workspace)."""
    for pr in probs:
        pr["fista"].reset_device()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=torch.cuda.Stream()):
        run_step_device(adj, probs, ch, lanes)
    return graph


def run_e2e(adj, torch, probs, ch, out_host, lanes, steps):
    """`steps` steps through the public API with host buffers: every step's
    inputs (the three observations b and the channel batch s, h, x) are copied
    in from pinned host memory and its results (the LL bands of x and grad_h)
    read back.  The inputs are double-buffered: two copy streams bring step
    k + 1's inputs while step k computes, so the copies overlap the kernels
    (each step still copies all of its own inputs)."""
    main = torch.cuda.current_stream()
    css = lanes.copy_streams
    slots = lanes.e2e_slots
    for cs in css:
        cs.wait_stream(main)
    # two copy streams (two copy engines): s and the first observation on one,
    # x, h and the other observations on the other
    plan = [[("s", None), ("b", 0)], [("x", None), ("h", None)] + [("b", i) for i in range(1, len(probs))]]

    def copy_in(slot):
        for cs, items, ev in zip(css, plan, lanes.ev_in[slot]):
            with torch.cuda.stream(cs):
                for key, i in items:
                    if key == "b":
                        slots[slot]["b"][i].copy_(probs[i]["b_host"], non_blocking=True)
                    else:
                        slots[slot][key].copy_(ch[key + "_host"], non_blocking=True)
                ev.record(cs)

    copy_in(0)
    for k in range(steps):
        slot = k % 2
        if k + 1 < steps:
            if k >= 1:
                for cs in css:
                    cs.wait_event(lanes.ev_done[1 - slot])  # step k - 1 is done with that slot
            copy_in(1 - slot)
        lanes.fork()
        for st in lanes.streams:
            for ev in lanes.ev_in[slot]:
                st.wait_event(ev)
        for i, (pr, st) in enumerate(zip(probs, lanes.streams)):
            with torch.cuda.stream(st):
                pr["fista"].set_observation(slots[slot]["b"][i])
                pr["fista"].step(stream=st)
                ll = pr["wt"].band_rows[0] * pr["wt"].band_pitch[0]
                out_host["ll"][i, :ll].copy_(pr["fista"].x[:ll], non_blocking=True)
        st = lanes.streams[-1]
        with torch.cuda.stream(st):
            sl = slots[slot]
            adj.conv_gradient(sl["s"], sl["h"], sl["x"], grad_h=ch["gh"], grad_s=ch["gs"], ws=ch["ws"], stream=st)
            out_host["gh"].copy_(ch["gh"], non_blocking=True)
        lanes.join()
        lanes.ev_done[slot].record(main)
    for cs in css:
        main.wait_stream(cs)
    for pr in probs:  # back to the resident observation for the other measurements
        pr["fista"].set_observation(pr["b"])


def fista_time_to_tol(adj, torch, pr, tol=1e-4, ref_iters=3000, check_every=10, max_iters=3000):
    """Seconds for plain GPU FISTA from x0 = 0 to (F(x_k) - F*)/F* <= tol, checks included.
    F* = the smallest objective seen along a ref_iters-iteration run."""
    f = pr["fista"]
    f.reset()
    fstar = float("inf")
    for k in range(1, ref_iters + 1):
        val = f.step(objective=(k % 50 == 0 or k == ref_iters))
        if val is not None:
            fstar = min(fstar, val)
    f.reset()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    it, reached = 0, False
    while it < max_iters:
        it += 1
        val = f.step(objective=(it % check_every == 0))
        if val is not None and (val - fstar) / fstar <= tol:
            reached = True
            break
    torch.cuda.synchronize()
    return {"seconds": time.perf_counter() - t0, "iterations": it, "reached": reached, "F_star": fstar,
            "F_star_iterations": ref_iters, "check_every": check_every, "boundary": pr["bc"]}


def adjoint_vs_pinv(adj, torch, pr, iters=300):
    """F(x_k) after `iters` FISTA iterations with the exact adjoint W^* and with
    W^dagger in its place (the comparison the paper makes), same problem and L_f."""
    f = pr["fista"]
    g = adj.Fista(pr["wt"], pr["bl"], pr["b"], LAM, f.problem.lipschitz, gradient="pinv")
    f.reset()
    for _ in range(iters):
        f.step()
        g.step()
    fa, fp = f.objective(), g.objective()
    f.reset()
    return {"iterations": iters, "boundary": pr["bc"], "F_adjoint": fa, "F_pinv": fp, "ratio_pinv_over_adjoint": fp / fa}


def unrolled_gradient_timing(adj, torch, batch=16, size=512, levels=4, wavelet="db4", steps=10, reps=2):
    """The differentiation workload: a batch of `batch` problems of size^2,
    `levels`-level 8-tap Daubechies, symmetric boundaries, 9x9 Gaussian PSF
    sigma = 1.5 (the PSF of the 256^2 configuration; the workload names none),
    lambda = 1e-3; for each, `steps` FISTA iterations and the gradient of
    l = 1/2 ||W x_N - u||^2 with respect to (lambda, sigma, b) through them
    (checkpointed forward, recomputed segments, reverse mode).  Seconds for
    the whole batch, best of `reps`, forward alone and with the gradient."""
    from synthetic_inputs import gaussian_noise, piecewise_smooth_image, random_vector
    from paper_1707_02018_gb300.unrolled import UnrolledFista
    k, sigma = 9, 1.5
    p = gaussian_taps(k, sigma)
    runs = []
    for i in range(batch):
        seed = 9000 + i
        wt = adj.WtPlan(size, size, levels, wavelet, "sym")
        bl = adj.BlurPlan(size, size, p, p, "sym")
        img = wt.image(torch.as_tensor(piecewise_smooth_image(size, size, seed)))
        b = adj.blur(bl, img)
        b[:, :size] += torch.as_tensor(gaussian_noise((size, size), seed + 1, NOISE), dtype=torch.float32,
                                       device="cuda")
        f = adj.Fista(wt, bl, b, LAM, 1.0)
        L = f.lipschitz(wt.pack(random_vector(wt.logical_size, seed + 2)), iters=30)
        runs.append((UnrolledFista(size, size, levels, wavelet, "sym", k, sigma, "sym", b, LAM, L), img))
    for un, img in runs[:1]:
        un.grads(steps, img)  # warm-up (plans, allocations)
    fwd, full = [], []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for un, _ in runs:
            un.solve(steps)
        torch.cuda.synchronize()
        fwd.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        for un, img in runs:
            un.grads(steps, img)
        torch.cuda.synchronize()
        full.append(time.perf_counter() - t0)
    return {"batch": batch, "size": size, "levels": levels, "wavelet": wavelet, "boundary": "sym",
            "psf": [k, sigma], "steps": steps, "forward_sec": min(fwd), "gradient_sec": min(full),
            "gradient_over_forward": min(full) / min(fwd),
            "wrt": "lambda, sigma (Gaussian PSF width), b; checkpoints every floor(sqrt(steps)) iterations"}


# Batched solves: independent deblurring problems of uneven sizes, depths,
# wavelets and PSF widths (symmetric boundaries), all to the same relative
# objective tolerance.
BATCH_PROBLEMS = 24
BATCH_SIZES = (128, 256, 384, 512, 768, 1024)
BATCH_WAVELETS = ("db2", "db4", "cdf97")


def learned_warm_start(adj, torch, size=512, levels=4, wavelet="cdf97", n_train=48, n_test=4, target_iters=500,
                       batch=8, train_steps=600, lr=1e-3, tol=1e-4, check_every=10, ref_iters=3000, max_iters=3000):
    """The learned-warm-start workload: seeded size^2 problems (piecewise-smooth
    image, 9x9 Gaussian sigma 1.5 with symmetric boundaries, N(0, 1e-3) noise,
    `levels`-level CDF 9/7 with symmetric boundaries, lambda = 1e-3).  Targets:
    the images W x_500 of 500-iteration GPU FISTA solutions; the network is
    trained on them with the library's kernels (Adam, `train_steps` steps of
    `batch` images cycling over n_train problems); then, on n_test held-out
    problems, seconds and iterations of FISTA to (F - F*)/F* <= tol from zero
    and from x_0 = W^dagger u_hat (inference and W^dagger inside the timed
    region), F* the smallest objective of a ref_iters run; and the first
    checked zero-start iteration whose objective is at or below F(x_0) (the
    iterations the prediction stands for); and the held-out problems solved
    all at once (a CUDA graph of device-momentum iterations, a stream per
    problem) from zero and from the learned start, against the zero starts
    one after another (the metric's batched / batched + learned vs plain).
    The network and its training set are smaller than a production one
    (20,000 images): this measures the mechanism, not a tuned predictor."""
    from paper_1707_02018_gb300 import warmstart
    from synthetic_inputs import gaussian_noise, he_normal_params, piecewise_smooth_image, random_vector
    p = gaussian_taps(9, 1.5)
    wt = adj.WtPlan(size, size, levels, wavelet, "sym")
    bl = adj.BlurPlan(size, size, p, p, "sym")
    pitch = wt.image_pitch
    total = n_train + n_test
    B = torch.zeros(total, size, pitch, dtype=torch.float32, device="cuda")
    U = torch.zeros_like(B)
    t0 = time.perf_counter()
    L = None
    for i in range(total):
        seed = 11000 + i
        img = wt.image(torch.as_tensor(piecewise_smooth_image(size, size, seed)))
        adj.blur(bl, img, out=B[i])
        B[i, :, :size] += torch.as_tensor(gaussian_noise((size, size), seed + 1, NOISE), dtype=torch.float32,
                                          device="cuda")
        f = adj.Fista(wt, bl, B[i], LAM, 1.0)
        if L is None:  # the same operator A = R W for every problem
            L = f.lipschitz(wt.pack(random_vector(wt.logical_size, 12000)), iters=30)
        f.set_lipschitz(L)
        f.reset()
        for _ in range(target_iters):
            f.step()
        adj.wt_synth(wt, f.x, image=U[i])
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0

    net = warmstart.WarmStartNet(he_normal_params(warmstart.LAYER_SHAPES, 13000))
    nb = n_train // batch
    losses = []
    for k in range(3):  # warm-up (allocations, first launches)
        net.forward(B[:batch], size, size)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(train_steps):
        j = k % nb
        loss = net.train_step(B[j * batch:(j + 1) * batch], U[j * batch:(j + 1) * batch], size, size, lr=lr)
        if k % 100 == 0 or k == train_steps - 1:
            losses.append(float(loss))
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    # one traced step: per-kernel device times
    adj.trace_enable(512)
    adj.trace_reset()
    net.train_step(B[:batch], U[:batch], size, size, lr=0.0)
    torch.cuda.synchronize()
    recs = adj.trace_records()
    adj.trace_enable(0)
    per = {}
    for name, _, ms in recs:
        c, t = per.get(name, (0, 0.0))
        per[name] = (c + 1, t + ms)
    px = batch * size * size
    fwd = per.get("cnn_conv32_tc", (1, float("nan")))
    bwd = per.get("cnn_conv32_tc_bwd", (1, float("nan")))
    wgr = per.get("cnn_conv32_wgrad", (1, float("nan")))
    flop = 2.0 * 288 * 32 * px
    kern = {name: {"launches": c, "ms_total": t} for name, (c, t) in sorted(per.items())}
    conv = {"forward_us": 1e3 * fwd[1] / fwd[0], "data_grad_us": 1e3 * bwd[1] / bwd[0],
            "weight_grad_us": 1e3 * wgr[1] / wgr[0],
            "forward_GBps": 128.0 * px / (fwd[1] / fwd[0] * 1e-3) / 1e9,
            "data_grad_GBps": 192.0 * px / (bwd[1] / bwd[0] * 1e-3) / 1e9,
            "forward_TFLOPs": flop / (fwd[1] / fwd[0] * 1e-3) / 1e12,
            "weight_grad_TFLOPs": flop / (wgr[1] / wgr[0] * 1e-3) / 1e12,
            "bytes_per_pixel": {"forward": 128, "data_grad": 192}}
    pk = peaks()
    fwd_gbs = 128.0 * px / (fwd[1] / fwd[0] * 1e-3) / 1e9
    conv["roofline"] = {"kernel": "cnn_conv32_tc (forward)", "bound": "hbm", "achieved": fwd_gbs,
                        "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": fwd_gbs / pk["hbm_gbs"],
                        "traffic": NCU_TRAFFIC["cnn_conv32_tc"], "peak_source": pk["source"],
                        "algorithmic_bytes": 128 * px}

    def time_to_tol(f, x0, match=None):
        """(seconds, iterations, reached, first checked iteration with F <= match)."""
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if x0 is not None:
            x0 = x0()
        f.reset(x0)
        it, reached, matched = 0, False, None
        while it < max_iters:
            it += 1
            val = f.step(objective=(it % check_every == 0))
            if val is not None and match is not None and matched is None and val <= match:
                matched = it
            if val is not None and (val - fstar) / fstar <= tol:
                reached = True
                break
        torch.cuda.synchronize()
        return time.perf_counter() - t0, it, reached, matched

    tests = []
    for i in range(n_train, total):
        f = adj.Fista(wt, bl, B[i], LAM, L)
        f.reset()
        fstar = float("inf")
        for k in range(1, ref_iters + 1):
            val = f.step(objective=(k % 50 == 0 or k == ref_iters))
            if val is not None:
                fstar = min(fstar, val)
        nz_sol = float((f.x != 0).sum()) / f.x.numel()  # the ref_iters solution
        f0 = f.objective(torch.zeros_like(f.x))
        tau = LAM / L  # the threshold of one FISTA prox
        xd = net.warm_start(wt, B[i])            # dense: W^dagger u_hat
        xw = net.warm_start(wt, B[i], tau=tau)   # soft-thresholded at lambda / L
        fd, fw = f.objective(xd), f.objective(xw)
        nz = lambda v: float((v != 0).sum()) / v.numel()
        zs, zi, zr, zm = time_to_tol(f, None, match=fw)
        ws_, wi, wr, _ = time_to_tol(f, lambda: net.warm_start(wt, B[i], tau=tau))
        ds, di, dr, _ = time_to_tol(f, lambda: net.warm_start(wt, B[i]))
        tests.append({"F_star": fstar, "rel_F_at_zero": (f0 - fstar) / fstar, "rel_F_at_warm": (fw - fstar) / fstar,
                      "rel_F_at_warm_dense": (fd - fstar) / fstar, "nonzero_frac_warm": nz(xw),
                      "nonzero_frac_warm_dense": nz(xd), "nonzero_frac_fista_solution": nz_sol,
                      "zero_start_iterations_to_F_warm": zm,
                      "zero_start": {"seconds": zs, "iterations": zi, "reached": zr},
                      "warm_start": {"seconds": ws_, "iterations": wi, "reached": wr},
                      "warm_start_dense": {"seconds": ds, "iterations": di, "reached": dr}})
    zsum = sum(t["zero_start"]["seconds"] for t in tests)
    wsum = sum(t["warm_start"]["seconds"] for t in tests)
    dsum = sum(t["warm_start_dense"]["seconds"] for t in tests)

    # batched (+ learned): every held-out problem at once, a CUDA graph of
    # check_every device-momentum iterations per still-active problem (one
    # stream each) plus their objectives, replayed until all reach tol and
    # captured again over the rest as problems converge; from zero, and from
    # the learned start (inference inside the timed region)
    hold = list(range(n_train, total))
    fstar_h = np.array([t["F_star"] for t in tests])
    fs = [adj.Fista(wt, bl, B[i], LAM, L) for i in hold]
    sts = [torch.cuda.Stream() for _ in fs]
    objs = torch.zeros(len(fs), dtype=torch.float64, device="cuda")
    objs_host = torch.zeros(len(fs), dtype=torch.float64).pin_memory()
    for f, st in zip(fs, sts):  # kernel attributes, occupancy caches
        f.reset_device(stream=st)
        f.step_device(stream=st)
    torch.cuda.synchronize()

    def capture(active):
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=torch.cuda.Stream()):
            main = torch.cuda.current_stream()
            for i in active:
                sts[i].wait_stream(main)
            for i in active:
                for k in range(check_every):
                    fs[i].step_device(objective_out=objs[i:i + 1] if k == check_every - 1 else None, stream=sts[i])
            for i in active:
                main.wait_stream(sts[i])
        return graph

    def batched_solve(learned):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cur = torch.cuda.current_stream()
        for j, (f, st) in enumerate(zip(fs, sts)):
            x0 = net.warm_start(wt, B[hold[j]], tau=LAM / L) if learned else None
            st.wait_stream(cur)
            f.reset_device(x0, stream=st)
        active, it, caps = list(range(len(fs))), 0, 1
        graph = capture(active)
        while it < max_iters and active:
            graph.replay()
            it += check_every
            objs_host.copy_(objs)
            torch.cuda.synchronize()
            rel = (objs_host.numpy() - fstar_h) / fstar_h
            still = [i for i in active if rel[i] > tol]
            if still and len(still) < len(active):
                graph = capture(still)
                caps += 1
            active = still
        torch.cuda.synchronize()
        return {"seconds": time.perf_counter() - t0, "iterations": it, "reached": not active, "captures": caps}

    bz = batched_solve(False)
    bl_ = batched_solve(True)
    return {"size": size, "levels": levels, "wavelet": wavelet, "train_images": n_train, "test_images": n_test,
            "target_iterations": target_iters, "targets_sec": gen_s, "batch": batch, "train_steps": train_steps,
            "train_sec": train_s, "train_images_per_sec": train_steps * batch / train_s,
            "loss_every_100_steps": losses, "conv32": conv, "train_step_kernels": kern, "held_out": tests,
            "zero_start_sec_total": zsum, "warm_start_sec_total": wsum, "speedup": zsum / wsum,
            "warm_start": "x_0 = S_tau(W^dagger u_hat), tau = lambda / L (one prox threshold)",
            "dense_warm_start_sec_total": dsum, "speedup_dense": zsum / dsum,
            "batched_zero_start": bz, "batched_learned": bl_,
            "speedup_batched_vs_plain": zsum / bz["seconds"],
            "speedup_batched_learned_vs_plain": zsum / bl_["seconds"],
            "batched": "the held-out problems at once: one CUDA graph of device-momentum iterations per "
                       "still-active problem (a stream each), recaptured as problems converge; plain = "
                       "zero start, one problem after another (zero_start_sec_total)"}


def batch_problems(adj, torch, seed=7000):
    from synthetic_inputs import gaussian_noise, piecewise_smooth_image, random_vector
    rng = np.random.default_rng(seed)
    out = []
    for i in range(BATCH_PROBLEMS):
        n = int(rng.choice(BATCH_SIZES))
        J = int(rng.integers(3, 7))
        w = str(rng.choice(BATCH_WAVELETS))
        sigma = float(rng.uniform(0.8, 3.0))
        k = 2 * int(np.ceil(3 * sigma)) + 1
        p = gaussian_taps(k, sigma)
        wt = adj.WtPlan(n, n, J, w, "sym")
        bl = adj.BlurPlan(n, n, p, p, "sym")
        img = wt.image(torch.as_tensor(piecewise_smooth_image(n, n, seed + 10 * i)))
        b = adj.blur(bl, img)
        b[:, :n] += torch.as_tensor(gaussian_noise((n, n), seed + 10 * i + 1, NOISE), dtype=torch.float32,
                                    device="cuda")
        f = adj.Fista(wt, bl, b, LAM, 1.0)
        f.set_lipschitz(f.lipschitz(wt.pack(random_vector(wt.logical_size, seed + 10 * i + 2)), iters=20))
        out.append({"n": n, "J": J, "wavelet": w, "sigma": sigma, "fista": f, "wt": wt, "bl": bl, "b": b})
    return out


# The batching workload at its stated size: 512 problems, 150 iterations each.
CFG4_PROBLEMS, CFG4_ITERS = 512, 150


def cfg4_problems(adj, torch, count, seed=8000):
    """Seeded problems of the batching workload: square sizes U{128 ... 1024},
    levels U{3..6}, db2 / db4 / CDF 9/7, Gaussian PSF sigma U[0.8, 3] with
    2 ceil(3 sigma) + 1 taps, symmetric boundaries, lambda = 1e-3.  The step
    1/L_f uses L_f = 1.01 ||W||^2 >= ||R W||^2 (||R|| <= 1 for a normalised
    nonnegative PSF under symmetric boundaries), ||W||^2 by a 20-step power
    iteration on W^* W per (size, levels, wavelet)."""
    from synthetic_inputs import gaussian_noise, piecewise_smooth_image, random_vector
    rng = np.random.default_rng(seed)
    norms, out = {}, []
    for i in range(count):
        n = int(rng.choice(BATCH_SIZES))
        J = int(rng.integers(3, 7))
        w = str(rng.choice(BATCH_WAVELETS))
        sigma = float(rng.uniform(0.8, 3.0))
        k = 2 * int(np.ceil(3 * sigma)) + 1
        p = gaussian_taps(k, sigma)
        wt = adj.WtPlan(n, n, J, w, "sym")
        bl = adj.BlurPlan(n, n, p, p, "sym")
        key = (n, J, w)
        if key not in norms:
            v = wt.pack(random_vector(wt.logical_size, seed + 1))
            for _ in range(20):
                v = adj.wt_synth_adjoint(wt, adj.wt_synth(wt, v))
                nv = float(v.double().norm())
                v = v / nv
            norms[key] = nv
        img = wt.image(torch.as_tensor(piecewise_smooth_image(n, n, seed + 10 * i)))
        b = adj.blur(bl, img)
        b[:, :n] += torch.as_tensor(gaussian_noise((n, n), seed + 10 * i + 1, NOISE), dtype=torch.float32,
                                    device="cuda")
        f = adj.Fista(wt, bl, b, LAM, 1.01 * norms[key])
        out.append({"n": n, "J": J, "wavelet": w, "sigma": sigma, "fista": f})
    return out


def batch_engine_cfg4(adj, torch, count=CFG4_PROBLEMS, iters=CFG4_ITERS, check_every=10):
    """The batching workload as stated: `count` problems, `iters` FISTA
    iterations each, timed three ways on the same problems (CUDA events):
      * engine: the batched engine, ONE persistent launch for all iterations
        of all problems;
      * graph: the problems on their own streams, `check_every` device-momentum
        iterations of every problem captured in one CUDA graph and replayed;
      * plain: one problem after another, host-driven fista_step.
    Afterwards F(x_150) of every problem from the engine's objective launch is
    compared with the plain run's."""
    probs = cfg4_problems(adj, torch, count)
    fs = [p["fista"] for p in probs]
    t0 = time.perf_counter()
    batch = adj.FistaBatch(fs)
    create_s = time.perf_counter() - t0
    info = batch.info()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    # engine
    batch.reset()
    batch.run(2)  # warm-up
    batch.reset()
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record()
    batch.run(iters)
    e1.record()
    torch.cuda.synchronize()
    engine_ms = e0.elapsed_time(e1)
    F_engine = batch.objective().cpu().numpy().copy()
    status = adj.device_status()
    # graph of streams
    streams = [torch.cuda.Stream() for _ in fs]
    for f, st in zip(fs, streams):
        f.reset_device(stream=st)
        f.step_device(stream=st)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=torch.cuda.Stream()):
        main = torch.cuda.current_stream()
        for st in streams:
            st.wait_stream(main)
        for f, st in zip(fs, streams):
            for _ in range(check_every):
                f.step_device(stream=st)
        for st in streams:
            main.wait_stream(st)
    torch.cuda.synchronize()
    capture_s = time.perf_counter() - t0
    for f, st in zip(fs, streams):
        f.reset_device(stream=st)
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record()
    for _ in range(iters // check_every):
        graph.replay()
    e1.record()
    torch.cuda.synchronize()
    graph_ms = e0.elapsed_time(e1)
    del graph
    # plain
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for f in fs:
        f.reset()
        for _ in range(iters):
            f.step()
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    F_plain = np.array([f.objective() for f in fs])
    rel = np.abs(F_engine - F_plain) / F_plain
    px = sum(p["n"] * p["n"] for p in probs)
    return {"problems": count, "iterations": iters, "pixels": px,
            "sizes": {str(s): sum(1 for p in probs if p["n"] == s) for s in BATCH_SIZES},
            "engine_sec": engine_ms / 1e3, "graph_sec": graph_ms / 1e3, "plain_sec": plain_s,
            "engine_vs_plain": plain_s / (engine_ms / 1e3), "engine_vs_graph": graph_ms / engine_ms,
            "engine_launches": 1, "engine_items_per_iteration": info["items_per_iteration"],
            "engine_stages": info["stages"], "engine_ctas": info["ctas"], "engine_create_sec": create_s,
            "graph_capture_sec": capture_s,
            "F_engine_vs_plain_max_rel": float(rel.max()), "device_status": status,
            "mix": "sizes U{128..1024}, levels U{3..6}, db2/db4/cdf97, sigma U[0.8,3], SYM, lambda 1e-3"}


def batched_vs_plain(adj, torch, tol=1e-4, check_every=10, ref_iters=5000, max_iters=5000):
    """Wall seconds until every problem of the batch has (F(x_k) - F*)/F* <= tol:
    plain = one problem after another, host-driven fista_step with an objective
    check every `check_every` iterations; batched = all problems at once, one
    CUDA graph holding `check_every` device-momentum iterations of every
    still-active problem (a stream per problem) plus their objectives,
    replayed until all have converged; the graph is captured again over the
    remaining problems whenever a quarter of them have converged (capture
    time included).  F* = the smallest objective of a ref_iters-iteration run."""
    probs = batch_problems(adj, torch)
    P = len(probs)
    streams = [torch.cuda.Stream() for _ in probs]
    objs = torch.zeros(P, dtype=torch.float64, device="cuda")
    objs_host = torch.zeros(P, dtype=torch.float64).pin_memory()
    for pr, st in zip(probs, streams):  # warm-up: kernel attributes, occupancy caches
        pr["fista"].reset_device(stream=st)
        pr["fista"].step_device(stream=st)
    torch.cuda.synchronize()

    def capture(active):
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=torch.cuda.Stream()):
            main = torch.cuda.current_stream()
            for i in active:
                streams[i].wait_stream(main)
            for i in active:
                for it in range(check_every):
                    probs[i]["fista"].step_device(objective_out=objs[i:i + 1] if it == check_every - 1 else None,
                                                  stream=streams[i])
            for i in active:
                main.wait_stream(streams[i])
        return graph

    def reset_all():
        for pr, st in zip(probs, streams):
            pr["fista"].reset_device(stream=st)
        torch.cuda.synchronize()

    t0 = time.perf_counter()
    graph = capture(list(range(P)))
    torch.cuda.synchronize()
    build = time.perf_counter() - t0
    # F* per problem
    reset_all()
    fstar = np.full(P, np.inf)
    for _ in range(ref_iters // check_every):
        graph.replay()
        objs_host.copy_(objs)
        torch.cuda.synchronize()
        fstar = np.minimum(fstar, objs_host.numpy())
    # batched
    reset_all()
    t0 = time.perf_counter()
    active, in_graph = list(range(P)), P
    it, captures = 0, 1
    while it < max_iters and active:
        graph.replay()
        it += check_every
        objs_host.copy_(objs)
        torch.cuda.synchronize()
        rel = (objs_host.numpy() - fstar) / fstar
        active = [i for i in active if rel[i] > tol]
        if active and len(active) <= 0.75 * in_graph:
            graph = capture(active)
            in_graph = len(active)
            captures += 1
    batched = time.perf_counter() - t0
    batched_iters = it
    graph_reached = not active
    # engine: `check_every` iterations of every active problem per launch,
    # then the objective launch; rebuilt over the remaining problems when a
    # quarter of them have converged (creation time included)
    for pr in probs:
        pr["fista"].reset()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    active = list(range(P))
    batch = adj.FistaBatch([probs[i]["fista"] for i in active])
    batch.reset()
    in_batch, it_e, rebuilds = list(active), 0, 0
    while it_e < max_iters and active:
        batch.run(check_every)
        it_e += check_every
        F = batch.objective().cpu().numpy()
        rel = {i: (F[k] - fstar[i]) / fstar[i] for k, i in enumerate(in_batch)}
        active = [i for i in active if rel[i] > tol]
        if active and len(active) <= 0.75 * len(in_batch):
            # the new batch continues from each problem's state: x, y as they
            # are; the momentum t restarts at the value the engine had reached
            keep = [probs[i]["fista"] for i in active]
            saved = [(f.x.clone(), f.y.clone()) for f in keep]
            batch = adj.FistaBatch(keep)
            batch.reset()
            for f, (xs, ys) in zip(keep, saved):
                f.x.copy_(xs)
                f.y.copy_(ys)
            batch.set_momentum(it_e)
            in_batch = list(active)
            rebuilds += 1
    torch.cuda.synchronize()
    engine_s = time.perf_counter() - t0
    engine_iters = it_e
    engine_reached = not active
    # plain
    plain, iters = 0.0, []
    for i, pr in enumerate(probs):
        f = pr["fista"]
        f.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        k = 0
        while k < max_iters:
            k += 1
            val = f.step(objective=(k % check_every == 0))
            if val is not None and (val - fstar[i]) / fstar[i] <= tol:
                break
        torch.cuda.synchronize()
        plain += time.perf_counter() - t0
        iters.append(k)
    return {"problems": P, "sizes": [pr["n"] for pr in probs], "plain_sec": plain, "batched_sec": batched,
            "speedup": plain / batched, "plain_iterations": iters, "batched_iterations": batched_iters,
            "engine_sec": engine_s, "engine_speedup": plain / engine_s, "engine_iterations": engine_iters,
            "engine_reached": engine_reached, "engine_rebuilds": rebuilds,
            "reached": graph_reached and max(iters) < max_iters, "graph_build_sec": build, "graph_captures": captures,
            "tol": tol, "check_every": check_every, "F_star_iterations": ref_iters,
            "mix": "sizes U{128..1024}, levels U{3..6}, db2/db4/cdf97, sigma U[0.8,3], SYM"}


def ours(args):
    import torch
    import torch.distributed as dist

    import paper_1707_02018_gb300 as adj

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    adj.lib()
    probs, ch = build_workload(adj, torch, rank)
    torch.cuda.synchronize()
    lanes = Lanes(torch, len(probs) + 1)
    for _ in range(args.warmup):
        run_step(adj, probs, ch, lanes)
    torch.cuda.synchronize()

    graph = None
    if not args.no_graph:
        graph = capture_step(adj, torch, probs, ch, lanes)
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize()

    traced = min(args.steps, 20)
    stream = torch.cuda.current_stream()
    clock = ClockSampler(local)
    clock.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    for _ in range(args.steps):
        if graph is not None:
            graph.replay()
        else:
            run_step(adj, probs, ch, lanes)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    ms_local = e0.elapsed_time(e1)
    clocks = clock.stop()
    # per-kernel times: further steps, untimed, run serially with event pairs
    # around every kernel (the same kernels as a replayed step)
    adj.trace_enable(traced * 64)
    for _ in range(traced):
        run_step_device(adj, probs, ch) if graph is not None else run_step(adj, probs, ch)
    torch.cuda.synchronize()
    recs = adj.trace_records()
    adj.trace_enable(0)
    # whole operators: the same serial steps with one event pair per operator
    # call and none between its kernels (level 2), so that the launches inside
    # an operator overlap as they do untraced
    adj.trace_level(2)
    adj.trace_enable(traced * 16)
    for _ in range(traced):
        run_step_device(adj, probs, ch) if graph is not None else run_step(adj, probs, ch)
    torch.cuda.synchronize()
    op_recs = adj.trace_records()
    adj.trace_enable(0)
    adj.trace_level(1)
    spans = {"wt_synth": [], "wt_adjoint_prox": [], "blur_normal": []}
    for name, _, oms in op_recs:
        if name.startswith("op:") and name[3:] in spans:
            spans[name[3:]].append(oms)

    ms = max_over_ranks(torch, dist, ms_local, world, "cuda")
    bytes_step = step_bytes()
    value = whole_job_rate(bytes_step, args.steps, world, ms)

    # per-kernel device time from the traced steps
    per = {}
    for name, tag, kms in recs:
        key = (f"{name}.L{tag}" if name.startswith("wt_") else f"{name}.{tag}") if tag else name
        d = per.setdefault(key, [0, 0.0])
        d[0] += 1
        d[1] += kms
    launches_per_step = len([r for r in recs if not r[0].endswith("_reset")]) / traced  # memsets are not kernels
    # operators that run as several kernels, timed as their sum per call:
    # R^*(R u - b) = two TMA-staged passes; level 1 of W = the TMA kernel (full
    # tiles) plus, under SYM, the tiled kernel on the border tiles
    per_op = {}
    if "blur" in per and "blur_adjoint" in per and "blur_normal" not in per:
        per_op["blur_normal"] = [per["blur"][0], per["blur"][1] + per["blur_adjoint"][1]]
    for op in ("wt_synth.L1", "wt_adjoint_prox.L1"):
        tma = op.replace(".L1", "_tma.L1")
        if tma in per:
            per_op[op] = [per[tma][0], per[tma][1] + per.get(op, [0, 0.0])[1]]
    pk = peaks()
    fb = {bc: fista_bytes(bc) for bc in BCS}
    cb = channel_bytes()
    alg = {"wt_synth.L1": sum(fb[bc]["level1"]["wt_synth"] for bc in BCS) / 3,
           "wt_adjoint_prox.L1": sum(fb[bc]["level1"]["wt_adjoint_prox"] for bc in BCS) / 3,
           "blur_normal": fb["sym"]["blur_normal"], "conv_gradient": cb["conv_gradient"]}
    kernels = {}
    for key, (n, tot) in sorted(per.items(), key=lambda kv: -kv[1][1]):
        entry = {"launches_per_step": n / traced, "ms_per_launch": tot / n, "share": tot / sum(v[1] for v in per.values())}
        if key in alg and key not in per_op:
            entry["gbs"] = alg[key] / (tot / n * 1e-3) / 1e9
        kernels[key] = entry
    for key, (n, tot) in per_op.items():
        kernels[key + " (sum of passes)"] = {"calls_per_step": n / traced, "ms_per_call": tot / n,
                                             "gbs": alg[key] / (tot / n * 1e-3) / 1e9}
    top = max(per.items(), key=lambda kv: kv[1][1])[0]
    top_ms = per[top][1] / per[top][0]
    achieved = alg.get(top, 0.0) / (top_ms * 1e-3) / 1e9
    roof = {"kernel": top, "bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"], "traffic": NCU_TRAFFIC.get(top), "peak_source": pk["source"]}
    if top == "conv_gradient":
        # the dense sums run on the tensor cores (tcgen05 TF32 split three ways, warp MMA for grad_h):
        # at 24 useful flop per byte the roofline bound is HBM; the useful float32 rate is reported beside it
        roof["useful_tflops"] = cb["flops"] / (top_ms * 1e-3) / 1e12
    hbm_roofs = {}
    both = dict(per, **per_op)
    # whole operators (all five levels), per boundary and over the three
    for op, calls in spans.items():
        if op not in ("wt_synth", "wt_adjoint_prox") or len(calls) != len(probs) * traced:
            continue
        tot_b, tot_ms = 0.0, 0.0
        for i, pr in enumerate(probs):
            ms_i = statistics.median(calls[i::len(probs)])
            b_i = fb[pr["bc"]][op]
            tot_b += b_i
            tot_ms += ms_i
            a = b_i / (ms_i * 1e-3) / 1e9
            hbm_roofs[f"{op}.whole.{pr['bc']}"] = {"ms": ms_i, "achieved_gbs": a, "frac_of_hbm": a / pk["hbm_gbs"]}
        a = tot_b / (tot_ms * 1e-3) / 1e9
        hbm_roofs[f"{op}.whole"] = {"ms": tot_ms / len(probs), "achieved_gbs": a, "frac_of_hbm": a / pk["hbm_gbs"],
                                    "how": "median device time of the whole call (all levels, launch gaps), one "
                                           "event pair per operator call in serial steps; algorithmic bytes "
                                           "C + N^2 + 2I (W) and 4C + N^2 + 2I (W^* + prox)"}
    if spans["blur_normal"]:  # R^*(R u - b) as one operator call (both passes, the gap between them)
        both["blur_normal"] = [1, statistics.median(spans["blur_normal"])]
    for key in ("wt_synth.L1", "wt_adjoint_prox.L1", "blur_normal", "conv_gradient"):
        if key in both:
            a = alg[key] / (both[key][1] / both[key][0] * 1e-3) / 1e9
            hbm_roofs[key] = {"achieved_gbs": a, "frac_of_hbm": a / pk["hbm_gbs"]}
    # float32 ceilings: the measured FMA rate of this GPU; R^*(R u - b) does
    # 2 flop per tap per pass, two separable passes each for R and R^*
    fma_tflops = adj.fp32_fma_peak()
    if "blur_normal" in hbm_roofs:
        blur_flops = 2 * 2 * 2 * PSF_K * SIZE * SIZE
        t = blur_flops / (both["blur_normal"][1] / both["blur_normal"][0] * 1e-3) / 1e12
        hbm_roofs["blur_normal"].update({"fp32_tflops": t, "frac_of_fp32": t / fma_tflops})
    if "conv_gradient" in hbm_roofs:
        t = cb["flops"] / (both["conv_gradient"][1] / both["conv_gradient"][0] * 1e-3) / 1e12
        hbm_roofs["conv_gradient"].update({"useful_tflops": t, "frac_of_fp32": t / fma_tflops})
    h2d_rate = pinned_h2d_rate(torch)

    # end to end through the public API with host buffers
    h2d = sum(pr["b_host"].numel() * 4 for pr in probs) + sum(ch[k + "_host"].numel() * 4 for k in ("s", "h", "x"))
    out_host = {"gh": torch.empty(CH_B, CH_K).pin_memory(),
                "ll": torch.empty(len(probs), max(p["wt"].band_rows[0] * p["wt"].band_pitch[0] for p in probs)).pin_memory()}
    d2h = out_host["gh"].numel() * 4 + sum(p["wt"].band_rows[0] * p["wt"].band_pitch[0] * 4 for p in probs)
    e2e_steps = max(3, min(args.steps, 50))
    lanes.copy_streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    lanes.ev_in = [[torch.cuda.Event(), torch.cuda.Event()] for _ in range(2)]
    lanes.ev_done = [torch.cuda.Event(), torch.cuda.Event()]
    lanes.e2e_slots = [{"b": [torch.empty_like(pr["b"]) for pr in probs],
                        **{key: torch.empty_like(ch[key]) for key in ("s", "h", "x")}} for _ in range(2)]
    run_e2e(adj, torch, probs, ch, out_host, lanes, 2)  # warm-up of the pipelined path
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    run_e2e(adj, torch, probs, ch, out_host, lanes, e2e_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(torch, dist, e0.elapsed_time(e1), world, "cuda")
    e2e_value = whole_job_rate(bytes_step, e2e_steps, world, e2e_ms)

    extra = {}
    if rank == 0 and not args.no_solve:
        extra["fista_sec_to_1e-4"] = fista_time_to_tol(adj, torch, probs[1])
        extra["fista_batched_vs_plain_to_1e-4"] = batched_vs_plain(adj, torch)
        extra["fista_batch_engine_512x150"] = batch_engine_cfg4(adj, torch)
        extra["fista_adjoint_vs_pinv"] = adjoint_vs_pinv(adj, torch, probs[1])
        extra["unrolled_fista_gradient"] = unrolled_gradient_timing(adj, torch)
        extra["learned_warm_start"] = learned_warm_start(adj, torch)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded piecewise-smooth images, N(0,1) signals)",
            "config": {"workload": WORKLOAD, "image": SIZE, "levels": LEVELS, "wavelet": WAVELET,
                       "boundaries": list(BCS), "psf": [PSF_K, PSF_SIGMA], "channels": [CH_B, CH_N, CH_K],
                       "parallelism": f"replicas x{world} (independent problems per rank)",
                       "l2": "inputs larger than L2: ~540 MB touched per step vs 129 MB L2",
                       "issue": ("CUDA graph of the step (three fista_step_device lanes + conv_gradient), "
                                 "replayed once per step" if graph is not None else "call by call on four streams"),
                       "bytes_per_step": bytes_step,
                       "level_kernels": {pr["bc"]: {"tma": pr["wt"].tma_levels(), "tma_ctas": pr["wt"].tma_ctas(),
                                                    "autotuned": AUTOTUNE}
                                         for pr in probs}},
            "roofline": roof, "hbm_rooflines": hbm_roofs, "kernels": kernels,
            "fp32_fma_peak_tflops": fma_tflops, "h2d_pinned_copy": h2d_rate,
            "e2e": {"value": e2e_value, "unit": "GB/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps,
                    "copies": "pinned host buffers; inputs double-buffered, step k+1's H2D on two copy streams "
                              "during step k's kernels; D2H of each step's results on its own streams"},
            "gpu_launches": int(round(launches_per_step * args.steps)), "clocks": clocks,
        }
        line.update(extra)
        if not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline(max_seconds=20.0)
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------------------ oracle (CPU) arm
def oracle_sample(rng_seed=0, boundaries=BCS, rows_conv=8):
    """One bounded sample of the step on the host with the float64 oracle:
    one FISTA iteration per listed boundary at 2048^2, plus the channel
    gradient of `rows_conv` of the 256 signals.  Returns (bytes, seconds)."""
    from oracle import conv as oconv
    from oracle import fista as ofista
    from synthetic_inputs import channel_problem, gaussian_noise, piecewise_smooth_image
    p = gaussian_taps(PSF_K, PSF_SIGMA)
    secs, nbytes = 0.0, 0
    for i, bc in enumerate(boundaries):
        img = piecewise_smooth_image(SIZE, SIZE, 2000 + i)
        b = img + gaussian_noise((SIZE, SIZE), 2001 + i, NOISE)
        prob = ofista.Problem(SIZE, SIZE, LEVELS, WAVELET, bc, p, p, bc, b, LAM)
        from oracle.layout import num_coeffs
        C = num_coeffs(SIZE, SIZE, LEVELS, 10, bc)
        x = np.zeros(C)
        t0 = time.perf_counter()
        ofista.fista_step(prob, x, x.copy(), 1.0, 1.0)
        secs += time.perf_counter() - t0
        nbytes += fista_bytes(bc)["total"]
    cp = channel_problem(rows_conv, CH_N, CH_K, seed=3000)
    x = oconv.conv_full(cp["h"], cp["s"]) + cp["noise"]
    t0 = time.perf_counter()
    r = oconv.conv_full(cp["h_est"], cp["s_est"]) - x
    oconv.conv_adjoint(cp["s_est"], cp["h_est"], r)
    secs += time.perf_counter() - t0
    nbytes += channel_bytes()["total"] * rows_conv // CH_B
    return nbytes, secs


def _oracle_task(task):
    """One piece of the step on one host core (a process of the pool): a FISTA
    iteration at 2048^2 for one boundary, or the channel gradient of a few
    signals.  Returns (bytes, compute start, compute end) on the wall clock."""
    kind, arg, seed = task
    from oracle import conv as oconv
    from oracle import fista as ofista
    from oracle.layout import num_coeffs
    from synthetic_inputs import channel_problem, gaussian_noise, piecewise_smooth_image
    if kind == "fista":
        bc = arg
        p = gaussian_taps(PSF_K, PSF_SIGMA)
        img = piecewise_smooth_image(SIZE, SIZE, 2000 + seed)
        b = img + gaussian_noise((SIZE, SIZE), 2001 + seed, NOISE)
        prob = ofista.Problem(SIZE, SIZE, LEVELS, WAVELET, bc, p, p, bc, b, LAM)
        x = np.zeros(num_coeffs(SIZE, SIZE, LEVELS, 10, bc))
        t0 = time.time()
        ofista.fista_step(prob, x, x.copy(), 1.0, 1.0)
        return fista_bytes(bc)["total"], t0, time.time()
    rows = arg
    cp = channel_problem(rows, CH_N, CH_K, seed=3000 + seed)
    x = oconv.conv_full(cp["h"], cp["s"]) + cp["noise"]
    t0 = time.time()
    r = oconv.conv_full(cp["h_est"], cp["s_est"]) - x
    oconv.conv_adjoint(cp["s_est"], cp["h_est"], r)
    return channel_bytes()["total"] * rows // CH_B, t0, time.time()


def _single_thread_env():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"


def oracle_pool(cores):
    """A pool of `cores` single-threaded oracle processes.  Spawned (never
    forked from a process that has touched the GPU) and warmed with one small
    task each, so imports stay outside the timed region."""
    import multiprocessing as mp
    _single_thread_env()
    pool = mp.get_context("spawn").Pool(cores, initializer=_single_thread_env)
    pool.map(_oracle_task, [("conv", 1, 99)] * cores)
    return pool


def oracle_parallel_sample(pool, cores, seed=0):
    """The step's pieces spread over `cores` processes: one FISTA iteration at
    2048^2 per core (boundaries in turn) and the channel gradient of 8
    signals per core.  Returns (bytes, wall seconds from the first compute
    start to the last compute end)."""
    tasks = [("fista", BCS[i % len(BCS)], seed + i) for i in range(cores)]
    tasks += [("conv", 8, seed + i) for i in range(cores)]
    res = pool.map(_oracle_task, tasks, chunksize=1)
    nbytes = sum(r[0] for r in res)
    return nbytes, max(r[2] for r in res) - min(r[1] for r in res)


def cpu_baseline(max_seconds=20.0):
    nbytes, secs = oracle_sample()
    out = {"value": nbytes / secs / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
           "sample": "one float64 FISTA iteration at 2048^2 for each of PER/SYM/ZERO + channel gradient of "
                     "8 of the 256 signals (numpy, single thread), bytes counted as on the GPU",
           "seconds": secs, "host_cores_available": os.cpu_count()}
    cores = os.cpu_count() or 1
    if cores > 1:
        pool = oracle_pool(cores)
        try:
            pb, ps = oracle_parallel_sample(pool, cores)
        finally:
            pool.close()
            pool.join()
        out["all_cores"] = {"value": pb / ps / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
                            "sample": f"{cores} single-threaded processes: one FISTA iteration at 2048^2 each "
                                      f"(PER/SYM/ZERO in turn) + channel gradient of 8 signals each",
                            "seconds": ps}
    return out


def reference(args, budget_s=150.0):
    """The oracle timed on all host cores: a pool of single-threaded
    processes (one per core) runs, each step, one FISTA iteration at 2048^2
    per core (PER, SYM, ZERO in turn) and the channel gradient of 8 signals
    per core; once the run has used `budget_s`, the remaining steps run the
    channel gradient of 8 signals per core only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    pool = oracle_pool(cores)
    times, total_bytes, spent = [], 0, 0.0
    try:
        for k in range(args.warmup + args.steps):
            if spent < budget_s:
                nbytes, secs = oracle_parallel_sample(pool, cores, seed=17 * k)
            else:
                res = pool.map(_oracle_task, [("conv", 8, 17 * k + i) for i in range(cores)], chunksize=1)
                nbytes, secs = sum(r[0] for r in res), max(r[2] for r in res) - min(r[1] for r in res)
            spent += secs
            if k >= args.warmup:
                times.append(secs)
                total_bytes += nbytes
    finally:
        pool.close()
        pool.join()
    secs = sum(times)
    value = total_bytes / secs / 1e9
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"per step on {cores} cores: one FISTA iteration at 2048^2 "
                   "per core (PER/SYM/ZERO in turn) + channel gradient of 8 of the 256 signals per core"},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle",
                         "sample": "float64 numpy oracle, one single-threaded process per host core, bounded "
                                   "sample per step"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def engine_sample(count, seed=8100):
    """The batched engine alone on `count` problems of the batching mix: run(2),
    run(5), objective(); prints the objectives and the device status."""
    import torch
    import paper_1707_02018_gb300 as adj
    probs = cfg4_problems(adj, torch, count, seed=seed)
    batch = adj.FistaBatch([p["fista"] for p in probs])
    batch.reset()
    batch.run(2)
    batch.run(5)
    F = batch.objective()
    torch.cuda.synchronize()
    print(json.dumps({"engine_sample": count, "objectives": [float(v) for v in F.cpu()],
                      "device_status": adj.device_status()}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline sample")
    ap.add_argument("--no-solve", action="store_true", help="skip the time-to-1e-4 solve")
    ap.add_argument("--autotune", action="store_true", help="measure the TMA / tiled kernel choice per wavelet level")
    ap.add_argument("--no-graph", action="store_true", help="time the step issued call by call, not a CUDA graph")
    ap.add_argument("--engine-sample", type=int, default=0, metavar="P",
                    help="only run the batched engine on P problems of the batching mix (two launches of the "
                         "iteration, then the objective launch) and exit: the profiling target of the engine")
    args = ap.parse_args()
    global AUTOTUNE
    AUTOTUNE = args.autotune
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.engine_sample:
        engine_sample(args.engine_sample)
        return
    if args.impl == "reference":
        reference(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
