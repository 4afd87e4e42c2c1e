"""Training and evaluation of the kernel-integral surrogate.

Host-side driver over the library's calls: every sample, forward, backward
and optimizer step runs in libsg's kernels; this module only decides which
bodies, batches and learning rates.

* ``collect_samples``: random bodies (spheres, tori, rounded boxes with random
  sizes, rotations and package counts), exact integrals on each, and the
  network-class points of every body (``Grid.surrogate_samples``),
  sub-sampled to a target count.
* ``train``: Adam with cosine decay over seeded random mini-batches.
* ``evaluate``: exact and surrogate integrals of one grid, their times and
  the surrogate's errors.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import MLP, Grid, SUR_CLASSES


def _torch():
    import torch
    return torch


def collect_samples(n_bodies=500, seed=4, target=20_000_000, p_lo=1e2, p_hi=1e5, reinit_iters=20, log=None):
    """Returns (x bf16 [n, 32], t float32 [n, 4], info) with n <= target:
    canonical inputs and targets of network-class points, each body's phi
    initialised from its distance and reinitialised `reinit_iters` sweeps
    (as the fields the surrogate later serves are)."""
    import sg_inputs as si
    torch = _torch()
    bodies = si.random_bodies(n_bodies, seed=seed, p_lo=p_lo, p_hi=p_hi)
    t0 = time.perf_counter()
    counts = []
    for shape, spec, _ in bodies:  # pass 1: how many candidates each body has
        g = Grid(spec)
        g.tag_allocate(shape)
        g.init_sdf(shape)
        if reinit_iters:
            g.reinit(reinit_iters, 0.5)
        g.kernel_integrals()
        counts.append(g.surrogate_samples(seed, keep=1.0, cap=0)[2])
        g.close()
    total = sum(counts)
    keep = min(1.0, target / max(total, 1))
    xs, ts = [], []
    n = 0
    for k, (shape, spec, _) in enumerate(bodies):  # pass 2: keep a hashed fraction
        g = Grid(spec)
        g.tag_allocate(shape)
        g.init_sdf(shape)
        if reinit_iters:
            g.reinit(reinit_iters, 0.5)
        g.kernel_integrals()
        x, t, _ = g.surrogate_samples(seed + k, keep=keep)
        xs.append(x)
        ts.append(t)
        n += x.shape[0]
        g.close()
    X = torch.cat(xs)[:target].contiguous()
    T = torch.cat(ts)[:target].contiguous()
    info = {"bodies": n_bodies, "candidates": int(total), "keep": keep, "samples": int(X.shape[0]),
            "seconds": time.perf_counter() - t0}
    if log:
        log("collected %d samples from %d candidates of %d bodies in %.1f s" % (X.shape[0], total, n_bodies,
                                                                                 info["seconds"]))
    return X, T, info


def train(net: MLP, X, T, steps=300_000, batch=16384, lr=3e-3, seed=4, log_every=0, log=None):
    """Adam with lr * (1 + cos(pi s / steps)) / 2 on seeded random batches
    (epochs of a seeded permutation).  The defaults are the production
    recipe: 300k steps of 16384 samples (about 8 s on one B300) take the
    h = 0.002 torus to a max abs error near 8e-4 after fallback.  Returns
    ([(step, loss)], seconds)."""
    torch = _torch()
    n = X.shape[0]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    per_epoch = max(1, n // batch)
    perm = None
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = []
    # the step call with its pointers formed once (the loop issues a step in
    # a few microseconds, below the step's device time)
    step_fn, h = net._lib.sg_mlp_train_step, net.handle
    xp, tp, lp = X.data_ptr(), T.data_ptr(), loss.data_ptr()
    t0 = time.perf_counter()
    for s in range(steps):
        b = s % per_epoch
        if b == 0:
            perm = torch.randperm(n, generator=gen, device="cuda").to(torch.int32)
            pp = perm.data_ptr()
        lr_s = lr * 0.5 * (1.0 + math.cos(math.pi * s / steps))
        want = log_every and (s % log_every == 0 or s == steps - 1)
        st = step_fn(h, batch, xp, tp, pp + 4 * b * batch, lr_s, lp if want else None)
        if st != 0:
            net._check(st)
        if want:
            hist.append((s, float(loss.item())))
            if log:
                log("step %d lr %.2e loss %.3e" % (s, lr_s, hist[-1][1]))
    torch.cuda.synchronize()
    return hist, time.perf_counter() - t0


def evaluate(g: Grid, net: MLP, reps=10):
    """Exact (mode 0) and surrogate (mode 1) integrals of grid g: times,
    errors of the surrogate against the exact values, class counts."""
    torch = _torch()
    fields = ("W", "Gx", "Gy", "Gz")
    Ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = Ev(), Ev()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t_exact = timed(lambda: g.kernel_integrals())
    exact = {f: g.field(f).clone() for f in fields}
    t_sur = timed(lambda: g.kernel_integrals(mode=1, mlp=net))
    cls = g.surrogate_classify()
    stats = g.surrogate_stats()
    net_pts = cls == 3
    err = {}
    for f in fields:
        d = (g.field(f) - exact[f]).abs()
        dn = d[net_pts]
        err[f] = {"max_abs": float(d.max()), "rms": float(d.pow(2).mean().sqrt()),
                  "max_abs_network_points": float(dn.max()) if dn.numel() else 0.0,
                  "p99_network_points": float(torch.quantile(dn[:1 << 24].float(), 0.99)) if dn.numel() else 0.0,
                  "frac_network_points_over_1e-3": float((dn > 1e-3).float().mean()) if dn.numel() else 0.0}
    active = sum(stats)
    return {"exact_ms": t_exact, "surrogate_ms": t_sur, "speedup": t_exact / t_sur,
            "classes": {k: v for k, v in zip(SUR_CLASSES, stats)},
            "fractions": {k: v / max(active, 1) for k, v in zip(SUR_CLASSES, stats)},
            "errors": err, "max_abs_error": max(e["max_abs"] for e in err.values())}
