#!/usr/bin/env python
"""Benchmark of the sparse-grid level-set hot path on one or more B300s.

Workload (per GPU): the torus (R = 0.6, r = 0.2) and the extruded triangular
prism, each on its own sparse grid at h = 0.002.  One step runs, for each
body: band tagging and package allocation, float-float level-set init,
gradient, 50 Godunov reinitialisation sweeps (CFL 0.5), exact kernel
integrals, and a Morton-ordered probe of 50M particles in the band.

Prints one JSON line.  ``value`` is cell-updates/s over the whole step (init,
gradient, each reinit sweep and the integrals each update every active data
point once; probe time counts in the denominator, probes are reported
separately).  ``--impl reference`` times the FP64 CPU oracle on a bounded
sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import sg_inputs as si  # noqa: E402

CFL = 0.5
BAND_HALF_WIDTH_CELLS = 2  # particles within +-2 coarse cells of the surface
HBM_FALLBACK_GBS = 6400.0


# ----------------------------------------------------------------------------
# host-side helpers (also exercised by the CPU multi-process tests)
# ----------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def combine_over_ranks(seconds: float, units: float, backend_device=None):
    """(max seconds over ranks, sum of units over ranks); identity at world 1."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return seconds, units
    dev = backend_device or "cpu"
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def partition_bodies(weights, world):
    """Independent bodies over `world` ranks by package count, greedy
    largest-first (each body, heaviest first, goes to the least-loaded rank;
    ties to the lower rank): no rank exchanges data with another.  The
    heaviest rank carries at most the mean load plus the heaviest body.
    Returns one list of body indices per rank, each in increasing order."""
    order = sorted(range(len(weights)), key=lambda i: (-float(weights[i]), i))
    loads = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (loads[k], k))
        parts[r].append(i)
        loads[r] += float(weights[i])
    return [sorted(p) for p in parts]


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return HBM_FALLBACK_GBS, "fallback"


def source_digest(*paths):
    h = hashlib.sha256()
    for path in paths:
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profile_traffic(kernel_files, summary):
    """DRAM traffic per launch from a committed ncu summary, or None when the
    kernel source changed since the counters were taken."""
    if isinstance(kernel_files, str):
        kernel_files = [kernel_files]
    p = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(p):
        return None
    fields = {}
    for line in open(p):
        if ":" in line and line.strip().startswith(("traffic_bytes_per_launch", "kernel_source_sha256_16",
                                                    "units_per_launch")):
            k, v = line.split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    if fields.get("kernel_source_sha256_16") != source_digest(*kernel_files):
        return None
    try:
        return float(fields["traffic_bytes_per_launch"]), float(fields.get("units_per_launch", "nan"))
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.path)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if r[5 + k].strip().lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# workload
# ----------------------------------------------------------------------------
def bodies_for(names, h):
    out = []
    for name in names:
        if name == "torus":
            shape, spec = si.torus_large(h)
        elif name == "prism":
            shape, spec = si.prism_large(h)
        elif name == "sphere_small":
            shape, spec = si.sphere_small()
        else:
            raise ValueError(name)
        out.append((name, shape, spec))
    return out


def particles_for(name, shape, spec, n, seed):
    w = BAND_HALF_WIDTH_CELLS * spec.lc
    jit = 0.5 * spec.h
    if name == "torus":
        return si.torus_band_particles(n, shape.p[0], shape.p[1], w, seed=seed, jitter=jit)
    if name == "prism":
        tri = ((shape.p[0], shape.p[1]), (shape.p[2], shape.p[3]), (shape.p[4], shape.p[5]))
        return si.prism_band_particles(n, tri, shape.p[6], shape.p[7], w, seed=seed, jitter=jit)
    return si.sphere_shell_particles(n, shape.p[0], 3 * spec.h, seed=seed)


class Body:
    def __init__(self, sg, torch, name, shape, spec, n_particles, seed, iters):
        self.name, self.shape, self.spec, self.iters = name, shape, spec, iters
        self.g = sg.Grid(spec)
        self.P = self.g.tag_allocate(shape)
        self.n_pt = 64 * (self.P - 2)
        x, y, z = particles_for(name, shape, spec, n_particles, seed)
        dev = [torch.from_numpy(v).cuda() for v in (x, y, z)]
        # the workload's particles are stored in Morton order (input preparation)
        _, order = self.g.morton_order(*dev)
        order = order.long()
        self.X = [v[order].contiguous() for v in dev]
        self.n = n_particles
        self.out = {k: torch.empty(n_particles, dtype=torch.float32, device="cuda") for k in sg.PROBE_OUTPUTS}
        self.host_x = None
        self.host_out = None

    def pin_host(self, torch):
        self.host_x = [v.cpu().pin_memory() for v in self.X]
        self.host_out = {k: torch.empty(self.n, dtype=torch.float32).pin_memory() for k in self.out}

    def run(self, ev=None, phases=None):
        g = self.g

        def mark(name):
            if ev is not None:
                e = ev()
                e.record()
                phases.append((self.name + ":" + name, e))

        mark("start")
        g.tag_allocate(self.shape)
        mark("tag")
        g.init_sdf(self.shape)
        mark("init")
        g.gradient()
        mark("gradient")
        g.reinit(self.iters, CFL)
        mark("reinit")
        g.kernel_integrals()
        mark("integrals")
        g.probe(*self.X, morton=True, out=self.out)
        mark("probe")

    def run_e2e(self, torch, stream, up, down, chunks=8):
        """One step from pinned host positions to pinned host outputs.  The
        grid part of the step (tag to integrals) needs no particles, so it runs
        on the body's stream (the grid is bound to it) while the positions go
        up on the upload stream; the probe then runs chunk by chunk (a chunk
        of Morton-ordered particles is itself in Morton order), each chunk's
        outputs going down on the download stream while the next is probed."""
        g, n = self.g, self.n
        cut = [n * i // chunks for i in range(chunks + 1)]
        arrived = []
        up.wait_stream(stream)  # the previous step's probe has read the positions
        with torch.cuda.stream(up):
            for i in range(chunks):
                a, b = cut[i], cut[i + 1]
                for d, h in zip(self.X, self.host_x):
                    d[a:b].copy_(h[a:b], non_blocking=True)
                e = torch.cuda.Event()
                e.record(up)
                arrived.append(e)
        with torch.cuda.stream(stream):
            g.tag_allocate(self.shape)
            g.init_sdf(self.shape)
            g.gradient()
            g.reinit(self.iters, CFL)
            g.kernel_integrals()
            stream.wait_stream(down)  # the previous step's outputs have gone down
            for i in range(chunks):
                a, b = cut[i], cut[i + 1]
                stream.wait_event(arrived[i])
                g.probe(*(v[a:b] for v in self.X), morton=True, out={k: v[a:b] for k, v in self.out.items()})
                e = torch.cuda.Event()
                e.record(stream)
                down.wait_event(e)
                with torch.cuda.stream(down):
                    for k, v in self.out.items():
                        self.host_out[k][a:b].copy_(v[a:b], non_blocking=True)


def sphere_with_packages(target):
    """Unit sphere on a grid whose band has about `target` packages
    (P ~ 4.6 area / lc^2, the same rule that sizes the random bodies)."""
    lc = math.sqrt(4.6 * 4.0 * math.pi / target)
    half = 1.0 + 4 * lc
    m = int(math.ceil(2 * half / lc))
    return si.sphere(1.0), si.GridSpec((-0.5 * m * lc,) * 3, (m, m, m), lc / 4.0)


def batch_section(sg, torch, n_bodies=256, iters=20, reps=5, seed=1):
    """256 random bodies (spheres, tori, rounded boxes; r ~ U[0.1, 1], random
    rotations, package counts log-uniform in [1e2, 1e5]) swept together by
    one autotuned batch plan, against one sphere of equal package count
    through the single-grid calls.  Both time the same sweeps per run:
    gradient, smoothed sign, `iters` reinit sweeps, exact integrals.  With
    several ranks the bodies are partitioned by package count
    (partition_bodies) and every rank runs its share as its own batch; times
    are the maximum over ranks, points the sum."""
    ws, rank, _ = dist_env()
    bodies = si.random_bodies(n_bodies, seed=seed)
    mine = partition_bodies([t for _, _, t in bodies], ws)[rank] if ws > 1 else list(range(n_bodies))
    grids = []
    for b in mine:
        shape, spec, _ = bodies[b]
        g = sg.Grid(spec)
        g.tag_allocate(shape)
        g.init_sdf(shape)
        grids.append(g)
    batch = sg.Batch(grids)
    P_tot = batch.P
    n_pt = 64 * sum(g.P - 2 for g in grids)
    for g in grids:
        g.close()
    plan, times = batch.autotune(sg.make_plan(reinit_iterations=iters, cfl=CFL), reps=2)
    Ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    batch.run(plan)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = Ev(), Ev()
    e0.record()
    for _ in range(reps):
        batch.run(plan)
    e1.record()
    torch.cuda.synchronize()
    batch_ms = e0.elapsed_time(e1) / reps
    batch.close()
    sweeps = iters + 2
    b_sec, b_pts = combine_over_ranks(batch_ms * 1e-3, float(n_pt), "cuda")

    shape, spec = sphere_with_packages(P_tot)
    g = sg.Grid(spec)
    P1 = g.tag_allocate(shape)
    g.init_sdf(shape)

    def single():
        g.gradient()
        g.reinit(iters, CFL)
        g.kernel_integrals()

    single()
    torch.cuda.synchronize()
    barrier()
    e0.record()
    for _ in range(reps):
        single()
    e1.record()
    torch.cuda.synchronize()
    single_ms = e0.elapsed_time(e1) / reps
    n1 = 64 * (P1 - 2)
    g.close()
    s_sec, s_pts = combine_over_ranks(single_ms * 1e-3, float(n1), "cuda")
    b_rate = b_pts * sweeps / b_sec
    s_rate = s_pts * sweeps / s_sec
    out = {"bodies": n_bodies, "packages": P_tot, "points": n_pt, "sweeps_per_run": sweeps,
           "plan": {"pkgs_per_item": plan.pkgs_per_item, "depth": plan.depth},
           "autotune_ms": {"%d,%d" % k: v for k, v in times.items()},
           "run_ms": batch_ms, "cell_updates_per_s": b_rate,
           "single_body": {"packages": P1, "points": n1, "run_ms": single_ms, "cell_updates_per_s": s_rate},
           "batch_over_single": b_rate / s_rate}
    if ws > 1:
        out["partition"] = {"ranks": ws, "rule": "greedy largest-first by target package count, no collective",
                            "bodies_rank0": len(mine) if rank == 0 else None, "run_ms_max_over_ranks": 1e3 * b_sec}
    return out


def consistency_section(sg, torch, reps=3, frac=0.2, seed=17):
    """Consistency (sign) correction on the h = 0.002 torus after synthetic
    sign noise: in 20% of the packages every value at |phi| >= 2h flips sign
    and 20% of the far cells swap inside <-> outside.  The noisy phi and cell
    table are restored between timed calls (outside the timed region)."""
    shape, spec = si.torus_large()
    g = sg.Grid(spec)
    P = g.tag_allocate(shape)
    g.init_sdf(shape)
    clean = g.field("phi").clone()
    pk, cells = si.sign_noise_masks(P, spec.n_cells, seed=seed, frac_pkg=frac, frac_cell=frac)
    phi, cp = g.field("phi"), g.field("cell_pkg")
    flip = torch.from_numpy(pk).cuda()[:, None] & (phi.abs() >= 2.0 * spec.h)
    phi[flip] = -phi[flip]
    far = torch.from_numpy(cells).cuda() & (cp < 2)
    cp[far] = 1 - cp[far]
    noisy_phi, noisy_cp = phi.clone(), cp.clone()
    Ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    ms, out = [], None
    for r in range(reps + 1):
        phi.copy_(noisy_phi)
        cp.copy_(noisy_cp)
        e0, e1 = Ev(), Ev()
        e0.record()
        out = g.consistency_correct(1.0)
        e1.record()
        torch.cuda.synchronize()
        if r:
            ms.append(e0.elapsed_time(e1))
    restored = bool(torch.equal(g.field("phi"), clean))
    n_pt = 64 * (P - 2)
    t = sum(ms) / len(ms)
    g.close()
    return {"workload": "torus (R 0.6, r 0.2) at h = 0.002, sign noise in %d%% of packages (|phi| >= 2h) and of far "
                        "cells, trust band |phi| < h" % int(100 * frac),
            "packages": P, "points": n_pt, "cells": spec.n_cells, "ms": t,
            "points_flipped": out[0], "far_cells_moved": out[1], "point_sweeps": out[2], "cell_sweeps": out[3],
            "restored_bit_exact": restored,
            "point_sweep_updates_per_s": n_pt * out[2] / (t * 1e-3)}


def multires_section(sg, torch, reps=3):
    """Multi-resolution initialisation of the shelled sphere at h = 1/1024:
    a stack of six layers from 8^3 coarse cells, each tagged from the one
    below (distances only under coarse core cells) and initialised, against
    tagging and initialising the finest layer in full.  Both include grid
    creation; times are wall-clock around synchronised device work."""
    shape, spec = si.shelled_sphere()
    L = sg.multires_layers(spec)

    def stack():
        M = sg.MultiResolution(spec, shape, layers=L)
        torch.cuda.synchronize()
        return M

    def full():
        g = sg.Grid(spec)
        g.tag_allocate(shape)
        g.init_sdf(shape)
        torch.cuda.synchronize()
        return g

    out = {}
    for name, fn in (("layers", stack), ("full", full)):
        fn().close()
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            obj = fn()
            ts.append(time.perf_counter() - t0)
            if name == "layers":
                M = obj
                out["evaluated"] = M.evaluated
                out["packages"] = [g.P for g in M.grids]
            obj.close()
        out[name + "_ms"] = 1e3 * min(ts)
    return {"workload": "shelled sphere (centre 0.5, radii 0.3 / 0.31) at h = 1/1024, %d layers" % L,
            "layers": L, "cells_finest": spec.n_cells, **out,
            "distance_evaluations_layers": int(sum(out["evaluated"])), "distance_evaluations_full": spec.n_cells}


def large_section(sg, torch, reps=3):
    """The bodies at the finer spacings that give about 3M packages each
    (torus h = 7e-4, prism h = 6e-4): each phase of the per-body chain timed
    with CUDA events, and the sweeps' achieved bandwidth by algorithmic bytes
    (reinit: 12 B per point + 32 B per package; gradient: 16 B per point +
    32 B per package; integrals: 20 B per point + 108 B per package)."""
    hbm, kind = measured_peaks()
    Ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def timed(fn, n=reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = Ev(), Ev()
        e0.record()
        for _ in range(n):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    out = {}
    for name, (shape, spec) in (("torus", si.torus_large(h=7e-4)), ("prism", si.prism_large(h=6e-4))):
        g = sg.Grid(spec)
        t_tag = timed(lambda: g.tag_allocate(shape), 1)
        P = g.P
        n_pt = 64 * (P - 2)
        t_init = timed(lambda: g.init_sdf(shape))
        t_grad = timed(g.gradient)
        t_r50 = timed(lambda: g.reinit(50, CFL), 1)
        t_int = timed(g.kernel_integrals)
        # the call's 50 sweeps (the first also forms S0) and its two far fills
        sweep = t_r50 / 50
        r = {"h": spec.h, "packages": P, "points": n_pt, "cells": spec.n_cells, "tag_ms": t_tag, "init_ms": t_init,
             "gradient_ms": t_grad, "reinit50_ms": t_r50, "reinit_sweep_ms": sweep, "integrals_ms": t_int}
        for k, ms, b in (("reinit_sweep", sweep, 12 * n_pt + 32 * (P - 2)), ("gradient", t_grad, 16 * n_pt + 32 * (P - 2)),
                         ("integrals", t_int, 20 * n_pt + 108 * (P - 2))):
            gbs = b / (ms * 1e-3) / 1e9
            r[k + "_GBs"] = gbs
            r[k + "_hbm_frac_of_" + kind] = gbs / hbm
        r["reinit_cell_updates_per_s"] = n_pt / (sweep * 1e-3)
        out[name] = r
        g.close()
    return {"workload": "torus (R 0.6, r 0.2) at h = 7e-4 and prism at h = 6e-4: tag, init, gradient, 50 reinit "
                        "sweeps, exact integrals, per phase", **out}


def sort_segments(grids, X, offsets):
    """Input preparation: each body's segment of the device particles X put in
    its Morton order (the walk order of the relaxation)."""
    for b, g in enumerate(grids):
        s, e = int(offsets[b]), int(offsets[b + 1])
        if e > s:
            seg = [v[s:e] for v in X]
            _, order = g.morton_order(*seg)
            o = order.long()
            for v, sv in zip(X, seg):
                v[s:e] = sv[o]
            del o, order, seg


def relax_section(sg, torch, net, trained, n_particles=100_000_000, steps=50, n_bodies=64, reps=3, seed=1):
    """Grid-particle coupling at scale: the first 64 bodies of the 256-body
    batch (spheres, tori, rounded boxes), 10^8 particles near their surfaces
    (shares proportional to package counts, Morton order per body), one graph
    of [gradient, 20 reinit sweeps, surrogate integrals with fallback] + 50
    relaxation steps, each a probe of phi, n, W, G and a move by
    -0.1 h clip(phi/h, -1, 1) n.  Positions are restored between timed
    replays (outside the timed region)."""
    t0 = time.perf_counter()
    ws, rank, _ = dist_env()
    bodies = si.random_bodies(n_bodies, seed=seed)
    mine = partition_bodies([t for _, _, t in bodies], ws)[rank] if ws > 1 else list(range(n_bodies))
    grids = []
    for b in mine:
        shape, spec, _ = bodies[b]
        g = sg.Grid(spec)
        g.tag_allocate(shape)
        g.init_sdf(shape)
        grids.append(g)
    x, y, z, off = si.relax_particles(bodies, n_particles, seed=5, subset=mine)
    n_mine = int(off[-1])
    gen_s = time.perf_counter() - t0
    X0 = [torch.from_numpy(v).cuda() for v in (x, y, z)]
    del x, y, z
    sort_segments(grids, X0, off)
    batch = sg.Batch(grids)
    P_tot = batch.P
    P_act = sum(g.P - 2 for g in grids)
    for g in grids:
        g.close()
    batch.set_surrogate(net)
    plan, _ = batch.autotune(sg.make_plan(reinit_iterations=20, cfl=CFL, integrals_mode=1), reps=1)
    X = [v.clone() for v in X0]
    out = {k: torch.empty_like(X[0]) for k in ("W", "Gx", "Gy", "Gz")}
    Ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def timed(sweeps):
        ms = []
        for r in range(reps + 1):  # the first call captures the graph and warms up
            batch.reset()
            for v, v0 in zip(X, X0):
                v.copy_(v0)
            torch.cuda.synchronize()
            barrier()
            e0, e1 = Ev(), Ev()
            e0.record()
            batch.relax(*X, off, steps, 0.1, plan=plan, sweeps=sweeps, out=out)
            e1.record()
            torch.cuda.synchronize()
            if r:
                ms.append(e0.elapsed_time(e1))
        return sum(ms) / len(ms)

    full_ms = timed(True)
    relax_ms = timed(False)
    full_s, pts = combine_over_ranks(full_ms * 1e-3, float(n_mine), "cuda")
    relax_s, _ = combine_over_ranks(relax_ms * 1e-3, float(n_mine), "cuda")
    full_ms, relax_ms = 1e3 * full_s, 1e3 * relax_s
    # moved distance after the 50 steps, a check that the run relaxed something
    moved = float(torch.sqrt(sum((a - b) ** 2 for a, b in zip(X, X0))).max())
    batch.close()
    step_ms = relax_ms / steps
    n_out = len(out)
    # this rank's algorithmic bytes of the call: the probe table packed once
    # (8 fields read, written), then one launch that takes every particle
    # through all the steps: positions read and written once, the n_out
    # outputs written, the fields the steps interpolate (phi, g and, for the
    # last step's outputs, W, G) read once
    pack_bytes = 64 * 64 * P_act
    relax_bytes = n_mine * (24 + 4 * n_out) + 32 * 64 * P_act
    alg_total = pack_bytes + relax_bytes
    hbm, kind = measured_peaks()
    achieved = alg_total / (relax_ms * 1e-3) / 1e9
    # the bound: 4-byte gathers served by L1, 32 per particle-step (8 corners
    # x phi, g; 64 in the last step), against one warp-wide load per SM and
    # clock (every lane's value in one 128-byte line), 148 SMs at the maximum
    # SM clock
    gathers = n_mine * (32 * (steps - 1) + 64)
    gather_peak = 148 * 32 * 2032e6
    return {"workload": "%d mixed bodies (first %d of the 256-body batch, seed %d), %d particles near their surfaces, "
                        "20 reinit sweeps + surrogate integrals with fallback, %d relaxation steps of 0.1 h, one graph"
                        % (n_bodies, n_bodies, seed, n_particles, steps),
            "packages": P_tot, "particles": n_particles, "steps": steps,
            "plan": {"pkgs_per_item": plan.pkgs_per_item, "depth": plan.depth},
            "surrogate_weights": "trained (surrogate section)" if trained else "random-init (surrogate not trained)",
            "graph_ms": full_ms, "relax_only_ms": relax_ms, "sweeps_ms": full_ms - relax_ms, "step_ms": step_ms,
            "particle_steps_per_s": pts * steps / (relax_ms * 1e-3),
            "pipeline_particle_steps_per_s": pts * steps / (full_ms * 1e-3),
            "partition": ({"ranks": ws, "rule": "greedy largest-first by target package count, no collective"}
                          if ws > 1 else None),
            "roofline": {"kernel": "k_batch_relax", "bound": "l1 gathers",
                         "achieved": gathers / (relax_ms * 1e-3) / 1e9, "peak": gather_peak / 1e9,
                         "unit": "Ggathers/s", "frac": gathers / (relax_ms * 1e-3) / gather_peak,
                         "peak_rule": "one warp-wide 4-byte load per SM and clock: 148 SMs x 32 lanes x 2032 MHz",
                         "hbm": {"achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                                 "peak_kind": kind, "algorithmic_bytes_per_call": alg_total,
                                 "bytes_rule": "probe table packed once (64 B per point), positions read and written "
                                               "once (24 B per particle), 4 B per output per particle, 32 B per "
                                               "point of fields read once"}},
            "max_displacement": moved, "setup_seconds": gen_s}


def surrogate_section(sg, torch, steps=300_000, batch=16384, samples=20_000_000):
    """Learned kernel integral: training samples from 500 random bodies
    (seed 4, 20 reinit sweeps, exact integrals as labels, in each point's
    canonical frame), `steps` Adam steps of `batch` samples on the library's
    own tensor-core kernels, then the exact and the surrogate integrals of
    the h = 0.002 torus after 50 reinit sweeps: times and errors."""
    from paper_2512_11473_b300 import surrogate as S
    X, T, info = S.collect_samples(target=samples)
    net = sg.MLP(si.mlp_init_params(4))
    hist, secs = S.train(net, X, T, steps=steps, batch=batch, log_every=steps // 4)
    del X, T
    shape, spec = si.torus_large()
    g = sg.Grid(spec)
    g.tag_allocate(shape)
    g.init_sdf(shape)
    g.reinit(50, CFL)
    r = S.evaluate(g, net)
    g.close()
    r["training"] = {"samples": info, "steps": steps, "batch": batch, "lr": 3e-3, "seconds": secs,
                     "loss": [[a, b] for a, b in hist]}
    return r, net


PAPER_TABLE1_MS = {  # "Performance Evaluation", Table 1 (units unstated; CPU unnamed)
    "sequential_1_thread": 22.948, "sequential_4_threads": 7.429,
    "stencil_1_thread": 59.972, "stencil_4_threads": 21.378,
}


def table1_section(sg, torch, reps=20):
    """The paper's Table 1 workload on the GPU: the shelled sphere at 1/1024,
    a sequential update of every active value (read + write 4 B per point)
    and the 7-point Laplacian (read 4 B, write 4 B per point, one face row
    per package)."""
    shape, spec = si.shelled_sphere()
    g = sg.Grid(spec)
    P = g.tag_allocate(shape)
    g.init_sdf(shape)
    n_pt = 64 * (P - 2)
    Ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    out = {}
    for name, fn, nbytes in (("sequential", lambda: g.sequential_update(1e-7), 8.0 * n_pt),
                             ("laplacian", g.laplacian, 8.0 * n_pt + 32.0 * (P - 2))):
        fn()
        torch.cuda.synchronize()
        e0, e1 = Ev(), Ev()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms": ms, "cell_updates_per_s": n_pt / (ms * 1e-3),
                     "achieved_GBs": nbytes / (ms * 1e-3) / 1e9}
    g.close()
    hbm, kind = measured_peaks()
    for v in out.values():
        v["hbm_frac_of_%s" % kind] = v["achieved_GBs"] / hbm
    return {"workload": "shelled sphere, centre (0.5, 0.5, 0.5), radii 0.3 / 0.31, h = 1/1024",
            "packages": P, "points": n_pt, "gpu": out, "paper_cpu_ms_context": PAPER_TABLE1_MS}


def phase_totals(phases):
    """Sum the durations between consecutive markers per phase name (ms)."""
    tot = {}
    for (n0, e0), (n1, e1) in zip(phases[:-1], phases[1:]):
        if n1.endswith(":start"):
            continue
        key = n1
        tot[key] = tot.get(key, 0.0) + e0.elapsed_time(e1)
    return tot


# ----------------------------------------------------------------------------
# oracle (CPU) samples
# ----------------------------------------------------------------------------
_PARTICLE_CACHE = {}


def oracle_sample(frac, iters, n_particles_full, seed=2):
    """Oracle pass over a spatial sample of the torus workload: the sub-domain
    x in [-1, -1 + 2 frac] of the h = 0.002 torus grid, the same per-point
    steps (tag/init, gradient, iters reinit sweeps, integrals), and a Morton
    sort plus probe of frac * n_particles_full band particles.
    Returns (cell_updates, probes, seconds, description)."""
    import oracle
    shape, spec = si.torus_large()
    nx = max(1, int(round(spec.dims[0] * frac)))
    sub = si.GridSpec(spec.lo, (nx, spec.dims[1], spec.dims[2]), spec.h)
    m = max(1000, int(n_particles_full * nx / spec.dims[0]))
    key = (m, seed)
    if key not in _PARTICLE_CACHE:
        _PARTICLE_CACHE.clear()
        _PARTICLE_CACHE[key] = particles_for("torus", shape, spec, m, seed)
    x, y, z = _PARTICLE_CACHE[key]
    t0 = time.perf_counter()
    G = oracle.build_grid(sub, shape)
    gx, gy, gz = oracle.gradient(sub, G.nbr, G.phi)
    phi = oracle.reinit(sub, G.nbr, G.phi, iters, CFL)
    W, Gx, Gy, Gz = oracle.kernel_integrals(sub, G.nbr, phi)
    keys = oracle.morton_keys(sub, x, y, z)
    order = oracle.morton_order(keys)
    oracle.probe(sub, G.cell_pkg, G.nbr, [phi, gx, gy, gz, W, Gx, Gy, Gz], x[order], y[order], z[order])
    secs = time.perf_counter() - t0
    n_pt = 64 * (G.P - 2)
    desc = ("torus h=0.002 sub-domain x in [-1, %.3f] (%d of %d cell columns, %d packages), %d reinit sweeps, "
            "%d probes" % (sub.lo[0] + nx * sub.lc, nx, spec.dims[0], G.P, iters, m))
    return n_pt * (iters + 3), m, secs, desc


def oracle_calibrate(iters, n_particles_full, frac=0.04):
    """Seconds the full oracle pass would take, extrapolated linearly from a
    small spatial sample."""
    _, _, secs, _ = oracle_sample(frac, iters, n_particles_full)
    return secs / frac


def cpu_threads():
    import oracle
    return oracle.get_threads()


# ----------------------------------------------------------------------------
# arms
# ----------------------------------------------------------------------------
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    est = oracle_calibrate(args.iters, args.particles)
    budget = max(5.0, 150.0 / max(1, args.steps + args.warmup))
    frac = min(1.0, max(0.02, budget / est))
    for _ in range(args.warmup):
        oracle_sample(frac, args.iters, args.particles)
    total_u, total_s, desc = 0.0, 0.0, ""
    for _ in range(args.steps):
        u, _, s, desc = oracle_sample(frac, args.iters, args.particles)
        total_u += u
        total_s += s
    value = total_u / total_s
    line = {"impl": "reference", "metric": "cell-updates/s", "value": value, "unit": "cell-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "torus+prism h=0.002, 50 reinit sweeps, exact integrals, 50M Morton probes "
                                   "per body (oracle: bounded spatial sample per step)", "sample": desc},
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": cpu_threads(), "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_sg(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2512_11473_b300 import build as sg_build
    sg_build.build()  # no-op unless a source is newer than libsg.so
    import paper_2512_11473_b300 as sg

    if args.only:
        # one side measurement on its own (for profiling it): no headline line
        if rank == 0:
            if args.only == "relax":
                net = sg.MLP(si.mlp_init_params(4))
                r = relax_section(sg, torch, net, False, n_particles=args.relax_particles,
                                  n_bodies=args.relax_bodies)
                net.close()
            elif args.only == "table1":
                r = table1_section(sg, torch)
            elif args.only == "consistency":
                r = consistency_section(sg, torch)
            elif args.only == "multires":
                r = multires_section(sg, torch)
            elif args.only == "large":
                r = large_section(sg, torch)
            else:
                r = batch_section(sg, torch, n_bodies=args.batch_bodies)
            print(json.dumps({"section": args.only, args.only: r}), flush=True)
        return 0

    names = args.bodies.split(",")
    bodies = [Body(sg, torch, n, s, sp, args.particles, 2 + k, args.iters)
              for k, (n, s, sp) in enumerate(bodies_for(names, args.h))]
    torch.cuda.synchronize()
    cell_updates = sum(b.n_pt * (args.iters + 3) for b in bodies)
    probes = sum(b.n for b in bodies)

    for _ in range(args.warmup):
        for b in bodies:
            b.run()
    torch.cuda.synchronize()
    barrier()

    Ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = sg.kernel_launch_count()
    phases = []
    torch.cuda.synchronize()
    barrier()
    t_start = Ev()
    t_start.record()
    torch.cuda.nvtx.range_push("timed_steps")  # lets a profiler list the timed launches alone
    for _ in range(args.steps):
        for b in bodies:
            b.run(Ev, phases)
    torch.cuda.nvtx.range_pop()
    t_end = Ev()
    t_end.record()
    torch.cuda.synchronize()
    barrier()
    launches = sg.kernel_launch_count() - launches0
    clk = clocks.stop()
    secs = t_start.elapsed_time(t_end) / 1e3
    tmax, units = combine_over_ranks(secs, cell_updates * args.steps, "cuda")
    value = units / tmax

    # per-phase breakdown (device events on the launching stream)
    tot = phase_totals(phases)
    breakdown = {k: v / args.steps for k, v in sorted(tot.items())}
    probe_ms = sum(v for k, v in breakdown.items() if k.endswith(":probe"))

    # dominant kernel: one reinit sweep, the step's reinit phase divided by
    # its sweeps (the first sweep also forms S0; the call's two far fills
    # stay in, so the figure errs low)
    sweep_ms = {b.name: breakdown[b.name + ":reinit"] / args.iters for b in bodies}
    big = max(bodies, key=lambda b: b.P)
    # read phi and S0, write phi (12 B per point) and the 32-byte face row
    # of every package
    alg_bytes = 12.0 * big.n_pt + 32.0 * (big.P - 2)
    # the same sweep by the per-point count of the scope table: 12 B per point
    # plus the 108-byte 27-entry neighbour row spread over the package's 64
    # points (1.7 B per point)
    alg_bytes_table = (12.0 + 108.0 / 64.0) * big.n_pt
    hbm, peak_kind = measured_peaks()
    achieved = alg_bytes / (sweep_ms[big.name] * 1e-3) / 1e9
    achieved_table = alg_bytes_table / (sweep_ms[big.name] * 1e-3) / 1e9
    csrc = os.path.join(ROOT, "paper_2512_11473_b300", "csrc")
    prof = profile_traffic([os.path.join(csrc, "sg_reinit.cu"), os.path.join(csrc, "sg_rows.cuh")],
                           "reinit_step_torus_h0.002.md")
    traffic = None
    if prof is not None:
        tb, units_prof = prof
        traffic = tb * (big.n_pt / units_prof) if units_prof == units_prof and units_prof > 0 else tb

    # the step's particles are stored in Morton order, so the probe's sort
    # check finds them sorted and skips the radix passes; the full sort of
    # the same particles in a shuffled order is timed here for reference
    big_b = max(bodies, key=lambda b: b.P)
    perm = torch.randperm(big_b.n, device="cuda")
    shuffled = [v[perm].contiguous() for v in big_b.X]
    del perm
    sort_ms = {}
    for label, pts in (("morton_ordered_input", big_b.X), ("shuffled_input", shuffled)):
        big_b.g.morton_order(*pts)
        e0, e1 = Ev(), Ev()
        e0.record()
        for _ in range(3):
            big_b.g.morton_order(*pts)
        e1.record()
        torch.cuda.synchronize()
        sort_ms[label] = e0.elapsed_time(e1) / 3
    del shuffled

    line = {
        "metric": "cell-updates/s", "value": value, "unit": "cell-updates/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tmax / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {
            "workload": "torus (R 0.6, r 0.2) + prism ((0,0),(1,0),(0.3,0.8) x [0,1]) at h=%g: tag/allocate, "
                        "init, gradient, %d reinit sweeps (CFL 0.5), exact kernel integrals, Morton probe of "
                        "%d particles per body" % (args.h, args.iters, args.particles),
            "bodies": {b.name: {"packages": b.P, "points": b.n_pt, "cells": b.spec.n_cells} for b in bodies},
            "cell_updates_per_step": cell_updates, "probes_per_step": probes,
            "l2": "inputs larger than L2: every reinit sweep streams >= 196 MB and a step touches several GB",
            "parallelism": "replicas (independent bodies per GPU, no collective)",
        },
        "probes_per_s": probes / (probe_ms * 1e-3) if probe_ms > 0 else None,
        "morton_sort_ms_%s_%dM" % (big.name, big.n // 1_000_000): sort_ms,
        "breakdown_ms_per_step": breakdown,
        "roofline": {"bound": "hbm", "kernel": "k_reinit_step (%s)" % big.name, "achieved": achieved,
                     "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "peak_kind": peak_kind,
                     "traffic": traffic, "algorithmic_bytes_per_launch": alg_bytes,
                     "bytes_rule": "12 B per point (read phi, S0; write phi) + 32 B per package (face row)",
                     "alt_bytes_rule": {"rule": "12 B + 108/64 B (27-entry row) per point",
                                        "algorithmic_bytes_per_launch": alg_bytes_table,
                                        "achieved": achieved_table, "frac": achieved_table / hbm},
                     "launch_ms": sweep_ms[big.name]},
        "gpu_launches": launches,
        "clocks": clk,
    }

    # end to end through the public API with host buffers
    if not args.no_e2e:
        for b in bodies:
            b.pin_host(torch)
        # one compute stream per body, one upload and one download stream: the
        # grid work overlaps the upload, the probe's chunks overlap the
        # download, and the two PCIe directions run concurrently; the span is
        # timed on the default stream, which starts them and waits for them
        main = torch.cuda.current_stream()
        streams = [torch.cuda.Stream() for _ in bodies]
        up, down = torch.cuda.Stream(), torch.cuda.Stream()
        torch.cuda.synchronize()
        for b, st in zip(bodies, streams):
            b.g.set_stream(st)
        for _ in range(max(1, min(args.warmup, 2))):
            for b, st in zip(bodies, streams):
                b.run_e2e(torch, st, up, down)
        torch.cuda.synchronize()
        barrier()
        e0, e1 = Ev(), Ev()
        e0.record(main)
        for st in streams + [up, down]:
            st.wait_stream(main)
        for _ in range(args.steps):
            for b, st in zip(bodies, streams):
                b.run_e2e(torch, st, up, down)
        for st in streams + [up, down]:
            main.wait_stream(st)
        e1.record(main)
        torch.cuda.synchronize()
        for b in bodies:
            b.g.set_stream(main)
        barrier()
        esecs, eunits = combine_over_ranks(e0.elapsed_time(e1) / 1e3, cell_updates * args.steps, "cuda")
        # the outputs that came down equal the device's (every 997th particle)
        same = all(torch.equal(b.host_out[k][::997], v[::997].cpu()) for b in bodies for k, v in b.out.items())
        line["e2e"] = {"value": eunits / esecs, "unit": "cell-updates/s",
                       "h2d_bytes_per_step": sum(12 * b.n for b in bodies),
                       "d2h_bytes_per_step": sum(4 * len(b.out) * b.n for b in bodies),
                       "outputs_match_device": bool(same)}
    line["table1"] = table1_section(sg, torch)
    if not args.no_consistency:
        line["consistency"] = consistency_section(sg, torch)
    if not args.no_multires:
        line["multires"] = multires_section(sg, torch)
    if not args.no_large:
        line["large"] = large_section(sg, torch)
    if not args.no_batch:
        line["batch"] = batch_section(sg, torch, n_bodies=args.batch_bodies)
    net = None
    if not args.no_surrogate:
        line["surrogate"], net = surrogate_section(sg, torch, steps=args.sur_steps)
    if not args.no_relax:
        trained = net is not None
        if net is None:
            net = sg.MLP(si.mlp_init_params(4))
        line["relax"] = relax_section(sg, torch, net, trained, n_particles=args.relax_particles,
                                      n_bodies=args.relax_bodies)
    if net is not None:
        net.close()
    if not args.no_cpu_baseline and rank == 0 and ws == 1:
        est = oracle_calibrate(args.iters, args.particles)
        frac = min(1.0, max(0.02, 15.0 / est))
        u, m, s, desc = oracle_sample(frac, args.iters, args.particles)
        line["cpu_baseline"] = {"value": u / s, "unit": "cell-updates/s", "cores": cpu_threads(), "kind": "oracle",
                                "sample": desc, "seconds": s}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["sg", "reference"], default="sg")
    ap.add_argument("--bodies", default="torus,prism")
    ap.add_argument("--h", type=float, default=0.002)
    ap.add_argument("--iters", type=int, default=50)
    ap.add_argument("--particles", type=int, default=50_000_000, help="probe particles per body")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 256-body batch measurement")
    ap.add_argument("--batch-bodies", type=int, default=256,
                    help="bodies in the batch measurement (the first n of the 256-body set)")
    ap.add_argument("--no-surrogate", action="store_true", help="skip training and timing the surrogate")
    ap.add_argument("--sur-steps", type=int, default=300_000,
                    help="Adam steps of the surrogate training (fewer only for profiling runs)")
    ap.add_argument("--no-relax", action="store_true", help="skip the 64-body particle relaxation")
    ap.add_argument("--relax-particles", type=int, default=100_000_000)
    ap.add_argument("--relax-bodies", type=int, default=64)
    ap.add_argument("--no-consistency", action="store_true", help="skip the sign-correction measurement")
    ap.add_argument("--no-multires", action="store_true", help="skip the multi-resolution measurement")
    ap.add_argument("--no-large", action="store_true", help="skip the ~3M-package bodies")
    ap.add_argument("--only", choices=["relax", "table1", "batch", "consistency", "multires", "large"],
                    help="run one side measurement alone and print it (no headline line)")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_sg(args)


if __name__ == "__main__":
    sys.exit(main())
