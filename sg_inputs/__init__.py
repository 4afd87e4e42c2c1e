"""Seeded synthetic inputs shared by the CPU oracle and the CUDA library.

This module holds no arithmetic of the sparse-grid method itself: no signed
distance evaluation, tagging, stencil or interpolation.  It only produces
*inputs*: shape descriptors, grid descriptors, random bodies and particle
positions, all drawn from one counter-based generator (SplitMix64, Steele,
Lea & Flood 2014) so that both sides see bit-identical data.

Shapes are described in a local frame: a world point x maps to the local
point q = R^T (x - centre), where ``rot`` is R stored row-major (local to
world).  Kinds and their parameter vector ``p``:

* SPHERE       p[0] = radius
* PLANE        the plane q_z = 0 (normal = third column of R); no parameters
* TORUS        p[0] = major radius (about the local z axis), p[1] = minor radius
* PRISM        p[0:6] = triangle (ax, ay, bx, by, cx, cy) in the local xy
               plane, extruded over q_z in [p[6], p[7]]
* ROUNDED_BOX  p[0:3] = half extents, p[3] = rounding radius
* SHELL        p[0] < p[1]: the solid between two concentric spheres
"""
from __future__ import annotations

import dataclasses
import math
import os

import numpy as np

SPHERE, PLANE, TORUS, PRISM, ROUNDED_BOX, SHELL = 0, 1, 2, 3, 4, 5
KIND_NAMES = {SPHERE: "sphere", PLANE: "plane", TORUS: "torus", PRISM: "prism",
              ROUNDED_BOX: "rounded_box", SHELL: "shell"}

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


# ----------------------------------------------------------------------------
# Generator
# ----------------------------------------------------------------------------
def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n outputs of SplitMix64 started at state ``seed``, skipping ``offset``.

    Counter form of the published generator: output k is mix(seed + (k+1)*gamma)
    with the two xor-shift-multiply rounds of Steele, Lea & Flood (2014).
    """
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class Stream:
    """Sequential view over one SplitMix64 sequence."""

    def __init__(self, seed: int):
        self.seed = int(seed)
        self.pos = 0

    def u64(self, n: int) -> np.ndarray:
        out = splitmix64(self.seed, n, self.pos)
        self.pos += n
        return out

    def uniform(self, n: int) -> np.ndarray:
        """Floats in [0, 1) from the top 24 bits (exact in float32)."""
        return (self.u64(n) >> np.uint64(40)).astype(np.float64) * (1.0 / (1 << 24))

    def uniform53(self, n: int) -> np.ndarray:
        """Doubles in [0, 1) from the top 53 bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


# ----------------------------------------------------------------------------
# Descriptors
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Shape:
    kind: int
    centre: tuple = (0.0, 0.0, 0.0)
    rot: tuple = (1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0)
    p: tuple = (0.0,) * 8

    def __post_init__(self):
        self.centre = tuple(float(v) for v in self.centre)
        self.rot = tuple(float(v) for v in self.rot)
        p = [float(v) for v in self.p] + [0.0] * 8
        self.p = tuple(p[:8])


@dataclasses.dataclass
class GridSpec:
    """Background mesh: dims coarse cells of size lc = 4h starting at lo.
    Optional: kernel_support (a length, 0 for 2h), heaviside_eps (a length,
    0 for h), id_order (0 linear cell order, 1 Morton order)."""
    lo: tuple
    dims: tuple
    h: float
    kernel_support: float = 0.0
    heaviside_eps: float = 0.0
    id_order: int = 0

    @property
    def lc(self) -> float:
        return 4.0 * self.h

    @property
    def n_cells(self) -> int:
        return int(self.dims[0]) * int(self.dims[1]) * int(self.dims[2])

    def hi(self):
        return tuple(self.lo[a] + self.dims[a] * self.lc for a in range(3))


def sphere(radius, centre=(0.0, 0.0, 0.0), rot=None) -> Shape:
    return Shape(SPHERE, centre, rot or Shape(SPHERE).rot, (radius,))


def plane(normal, point=(0.0, 0.0, 0.0)) -> Shape:
    """Plane through ``point`` whose local z axis is the unit ``normal``."""
    n = np.asarray(normal, dtype=np.float64)
    n = n / np.linalg.norm(n)
    a = np.array([1.0, 0.0, 0.0]) if abs(n[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = a - n * np.dot(a, n)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    R = np.stack([e1, e2, n], axis=1)  # columns: local axes in world frame
    return Shape(PLANE, point, tuple(R.reshape(-1)), ())


def torus(major, minor, centre=(0.0, 0.0, 0.0), rot=None) -> Shape:
    return Shape(TORUS, centre, rot or Shape(TORUS).rot, (major, minor))


def prism(tri, z0, z1, centre=(0.0, 0.0, 0.0), rot=None) -> Shape:
    (ax, ay), (bx, by), (cx, cy) = tri
    return Shape(PRISM, centre, rot or Shape(PRISM).rot, (ax, ay, bx, by, cx, cy, z0, z1))


def rounded_box(half, rounding, centre=(0.0, 0.0, 0.0), rot=None) -> Shape:
    return Shape(ROUNDED_BOX, centre, rot or Shape(ROUNDED_BOX).rot,
                 (half[0], half[1], half[2], rounding))


def shell(r_in, r_out, centre=(0.0, 0.0, 0.0)) -> Shape:
    return Shape(SHELL, centre, Shape(SHELL).rot, (r_in, r_out))


def quat_to_rot(q) -> tuple:
    """Row-major rotation matrix of the unit quaternion (w, x, y, z)."""
    w, x, y, z = q
    return (1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
            2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
            2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y))


def random_rotation(stream: Stream) -> tuple:
    """Uniform random rotation (Shoemake 1992, 'Uniform random rotations')."""
    u1, u2, u3 = stream.uniform53(3)
    a, b = math.sqrt(1.0 - u1), math.sqrt(u1)
    t2, t3 = 2.0 * math.pi * u2, 2.0 * math.pi * u3
    q = (b * math.cos(t3), a * math.sin(t2), a * math.cos(t2), b * math.sin(t3))
    return quat_to_rot(q)


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------
def _box_grid(lo, hi, h) -> GridSpec:
    lc = 4.0 * h
    dims = tuple(int(round((hi[a] - lo[a]) / lc)) for a in range(3))
    return GridSpec(tuple(float(v) for v in lo), dims, float(h))


def sphere_small():
    """Unit sphere at the origin in [-1.5, 1.5]^3 with h = 0.05 (15^3 cells)."""
    return sphere(1.0), _box_grid((-1.5,) * 3, (1.5,) * 3, 0.05)


def torus_large(h=0.002):
    """Torus R = 0.6, r = 0.2 about z in [-1,1]^2 x [-0.4,0.4]."""
    return torus(0.6, 0.2), _box_grid((-1.0, -1.0, -0.4), (1.0, 1.0, 0.4), h)


def shelled_sphere(h=1.0 / 1024):
    """The benchmark body of the paper's Table 1: a shell centred at
    (0.5, 0.5, 0.5) with radii 0.3 and 0.31, at resolution h in [0, 1]^3."""
    return shell(0.3, 0.31, (0.5, 0.5, 0.5)), _box_grid((0.0,) * 3, (1.0,) * 3, h)


PRISM_TRIANGLE = ((0.0, 0.0), (1.0, 0.0), (0.3, 0.8))


def prism_large(h=0.002):
    """Triangle (0,0),(1,0),(0.3,0.8) extruded over z in [0,1]."""
    return (prism(PRISM_TRIANGLE, 0.0, 1.0),
            _box_grid((-0.2, -0.2, -0.2), (1.2, 1.0, 1.2), h))


# ----------------------------------------------------------------------------
# Particle samplers (geometric sampling from shape parameters only)
# ----------------------------------------------------------------------------
def _unit_dirs(stream: Stream, n: int) -> np.ndarray:
    """Uniform directions: z uniform in [-1,1], azimuth uniform (Archimedes)."""
    z = 2.0 * stream.uniform53(n) - 1.0
    t = 2.0 * math.pi * stream.uniform53(n)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(t), s * np.sin(t), z], axis=1)


def sphere_shell_particles(n, radius, half_width, centre=(0.0, 0.0, 0.0), seed=0):
    """n points uniform in the shell radius-half_width < |x-c| < radius+half_width.

    For a sphere this shell is exactly the set |phi| < half_width.
    Returns float32 arrays x, y, z.
    """
    st = Stream(seed)
    d = _unit_dirs(st, n)
    r0, r1 = radius - half_width, radius + half_width
    r = np.cbrt(r0 ** 3 + st.uniform53(n) * (r1 ** 3 - r0 ** 3))
    pts = d * r[:, None] + np.asarray(centre)[None, :]
    return tuple(np.ascontiguousarray(pts[:, a], dtype=np.float32) for a in range(3))


def torus_band_particles(n, major, minor, half_width, seed=0, jitter=0.0):
    """n points uniform in the tube minor-w < dist(x, core circle) < minor+w.

    The volume element rho (major + rho cos v) drho dv du of the tube is sampled
    exactly: rho with density ~ rho, then acceptance (major + rho cos v)/(major + rho_max).
    Optional uniform jitter in [-jitter, jitter)^3 is added afterwards.
    """
    st = Stream(seed)
    out = []
    got = 0
    r0, r1 = minor - half_width, minor + half_width
    while got < n:
        m = int((n - got) * 1.4) + 1024
        rho = np.sqrt(r0 * r0 + st.uniform53(m) * (r1 * r1 - r0 * r0))
        v = 2.0 * math.pi * st.uniform53(m)
        u = 2.0 * math.pi * st.uniform53(m)
        acc = st.uniform53(m) * (major + r1) < (major + rho * np.cos(v))
        rho, v, u = rho[acc], v[acc], u[acc]
        s = major + rho * np.cos(v)
        pts = np.stack([s * np.cos(u), s * np.sin(u), rho * np.sin(v)], axis=1)
        out.append(pts)
        got += len(pts)
    pts = np.concatenate(out)[:n]
    if jitter > 0:
        pts = pts + (2.0 * st.uniform53(3 * n).reshape(n, 3) - 1.0) * jitter
    return tuple(np.ascontiguousarray(pts[:, a], dtype=np.float32) for a in range(3))


def prism_band_particles(n, tri, z0, z1, half_width, seed=0, jitter=0.0):
    """n points near the surface of an extruded triangle.

    A face is picked with probability proportional to its area (three side
    rectangles, two caps), a point uniform on that face, then an offset along
    the face normal uniform in [-half_width, half_width), then optional jitter.
    """
    st = Stream(seed)
    P = np.asarray(tri, dtype=np.float64)
    L = z1 - z0
    # orientation of the triangle (sign of twice its area)
    area2 = (P[1, 0] - P[0, 0]) * (P[2, 1] - P[0, 1]) - (P[1, 1] - P[0, 1]) * (P[2, 0] - P[0, 0])
    orient = 1.0 if area2 > 0 else -1.0
    edges = [(P[i], P[(i + 1) % 3]) for i in range(3)]
    areas = [np.linalg.norm(b - a) * L for a, b in edges] + [abs(area2) / 2] * 2
    cum = np.cumsum(areas) / np.sum(areas)
    f = np.searchsorted(cum, st.uniform53(n), side="right")
    a_, b_ = st.uniform53(n), st.uniform53(n)
    t = (2.0 * st.uniform53(n) - 1.0) * half_width
    pts = np.zeros((n, 3))
    for k, (a, b) in enumerate(edges):
        m = f == k
        e = b - a
        nrm = np.array([e[1], -e[0]]) * orient / np.linalg.norm(e)  # outward
        xy = a[None, :] + a_[m, None] * e[None, :] + t[m, None] * nrm[None, :]
        pts[m, 0:2] = xy
        pts[m, 2] = z0 + b_[m] * L
    for k, (zc, sgn) in ((3, (z0, -1.0)), (4, (z1, 1.0))):
        m = f == k
        s, r = a_[m], b_[m]
        flip = s + r > 1.0
        s = np.where(flip, 1.0 - s, s)
        r = np.where(flip, 1.0 - r, r)
        xy = P[0][None, :] + s[:, None] * (P[1] - P[0])[None, :] + r[:, None] * (P[2] - P[0])[None, :]
        pts[m, 0:2] = xy
        pts[m, 2] = zc + sgn * t[m]
    if jitter > 0:
        pts = pts + (2.0 * st.uniform53(3 * n).reshape(n, 3) - 1.0) * jitter
    return tuple(np.ascontiguousarray(pts[:, a], dtype=np.float32) for a in range(3))


def rounded_box_band_particles(n, half, rounding, half_width, seed=0, jitter=0.0):
    """n points near the surface of a rounded box (local frame, float64).

    The surface is split into its 6 flat faces, 12 quarter-cylinder edges and
    8 sphere-octant corners of the core box with half extents half - rounding;
    a piece is picked with probability proportional to its area, a point
    uniform on it, then an offset along its outward normal uniform in
    [-half_width, half_width), then optional jitter in [-jitter, jitter)^3.
    Returns an (n, 3) array.
    """
    st = Stream(seed)
    rho = float(rounding)
    a = np.asarray(half, dtype=np.float64) - rho
    pieces = []  # (kind, axis, signs)
    areas = []
    for i in range(3):
        j, k = (i + 1) % 3, (i + 2) % 3
        for s in (-1.0, 1.0):
            pieces.append(("face", i, (s,)))
            areas.append(4.0 * a[j] * a[k])
    for i in range(3):
        for sj in (-1.0, 1.0):
            for sk in (-1.0, 1.0):
                pieces.append(("edge", i, (sj, sk)))
                areas.append(math.pi * rho * a[i])
    for s0 in (-1.0, 1.0):
        for s1 in (-1.0, 1.0):
            for s2 in (-1.0, 1.0):
                pieces.append(("corner", 0, (s0, s1, s2)))
                areas.append(0.5 * math.pi * rho * rho)
    cum = np.cumsum(areas) / np.sum(areas)
    f = np.minimum(np.searchsorted(cum, st.uniform53(n), side="right"), len(pieces) - 1)
    u1, u2 = st.uniform53(n), st.uniform53(n)
    dirs = np.abs(_unit_dirs(st, n))
    t = (2.0 * st.uniform53(n) - 1.0) * half_width
    # per-piece tables: kind (0 face, 1 edge, 2 corner), axis, signs
    kind = np.array([("face", "edge", "corner").index(pc[0]) for pc in pieces])
    axis = np.array([pc[1] for pc in pieces])
    sgn = np.array([tuple(pc[2]) + (1.0,) * (3 - len(pc[2])) for pc in pieces])
    q = np.zeros((n, 3))
    nrm = np.zeros((n, 3))
    kf = kind[f]
    r = np.nonzero(kf == 0)[0]  # faces
    if r.size:
        i = axis[f[r]]
        j, k = (i + 1) % 3, (i + 2) % 3
        sv = sgn[f[r], 0]
        q[r, i] = sv * (a[i] + rho)
        q[r, j] = (2.0 * u1[r] - 1.0) * a[j]
        q[r, k] = (2.0 * u2[r] - 1.0) * a[k]
        nrm[r, i] = sv
    r = np.nonzero(kf == 1)[0]  # edges
    if r.size:
        i = axis[f[r]]
        j, k = (i + 1) % 3, (i + 2) % 3
        sj, sk = sgn[f[r], 0], sgn[f[r], 1]
        th = 0.5 * math.pi * u2[r]
        nrm[r, j] = sj * np.cos(th)
        nrm[r, k] = sk * np.sin(th)
        q[r, i] = (2.0 * u1[r] - 1.0) * a[i]
        q[r, j] = sj * a[j] + rho * nrm[r, j]
        q[r, k] = sk * a[k] + rho * nrm[r, k]
    r = np.nonzero(kf == 2)[0]  # corners
    if r.size:
        sv = sgn[f[r]]
        nrm[r] = sv * dirs[r]
        q[r] = sv * a[None, :] + rho * nrm[r]
    pts = q + t[:, None] * nrm
    if jitter > 0:
        pts = pts + (2.0 * st.uniform53(3 * n).reshape(n, 3) - 1.0) * jitter
    return pts


def body_band_particles(shape: Shape, n, half_width, seed=0, jitter=0.0):
    """n points near the surface of a sphere, torus or rounded box, sampled in
    the body's own frame (sphere: uniform in the shell |phi| < half_width;
    torus: uniform in the tube band; rounded box: surface point plus normal
    offset) and carried to the world frame x = centre + R q.  Returns float32
    arrays x, y, z."""
    if shape.kind == SPHERE:
        loc = np.stack(sphere_shell_particles(n, shape.p[0], half_width, seed=seed), axis=1).astype(np.float64)
        if jitter > 0:
            loc = loc + (2.0 * Stream(seed + 0x9E37).uniform53(3 * n).reshape(n, 3) - 1.0) * jitter
    elif shape.kind == TORUS:
        loc = np.stack(torus_band_particles(n, shape.p[0], shape.p[1], half_width, seed=seed, jitter=jitter),
                       axis=1).astype(np.float64)
    elif shape.kind == ROUNDED_BOX:
        loc = rounded_box_band_particles(n, shape.p[0:3], shape.p[3], half_width, seed=seed, jitter=jitter)
    else:
        raise ValueError("no band sampler for kind %d" % shape.kind)
    R = np.asarray(shape.rot, dtype=np.float64).reshape(3, 3)
    w = loc @ R.T + np.asarray(shape.centre)[None, :]
    return tuple(np.ascontiguousarray(w[:, a], dtype=np.float32) for a in range(3))


def relax_particles(bodies, n_total, seed=5, band_cells=2.0, jitter_h=0.5, subset=None):
    """Particles of a batch relaxation: n_total points over the bodies of
    ``random_bodies``, body b getting a share proportional to its target
    package count (so particles per package are about equal), sampled by
    ``body_band_particles`` with half-width band_cells coarse cells, jitter
    jitter_h fine cells and seed seed + b, stored body after body.
    subset: indices of the bodies to generate (their shares stay those of the
    whole set, so that the bodies of a partition get the particles they have
    in the whole run).  Returns (x, y, z, offsets) with offsets[k] the first
    particle of the k-th generated body."""
    tgt = np.array([t for _, _, t in bodies], dtype=np.float64)
    share = np.floor(n_total * tgt / tgt.sum()).astype(np.int64)
    rest = int(n_total - share.sum())
    share[:rest] += 1
    which = list(range(len(bodies))) if subset is None else [int(b) for b in subset]
    offsets = np.zeros(len(which) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(share[which])
    out = [np.empty(int(offsets[-1]), dtype=np.float32) for _ in range(3)]

    def one(k):  # bodies draw from their own streams: any schedule gives the same arrays
        b = which[k]
        shape, spec, _ = bodies[b]
        v = body_band_particles(shape, int(share[b]), band_cells * spec.lc, seed=seed + b, jitter=jitter_h * spec.h)
        for a in range(3):
            out[a][offsets[k]:offsets[k + 1]] = v[a]

    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        list(ex.map(one, range(len(which))))
    return out[0], out[1], out[2], offsets


def sign_noise_masks(P, n_cells, seed=6, frac_pkg=0.2, frac_cell=0.2):
    """Synthetic sign noise for the consistency correction, standing in for
    the wrong inside/outside decisions of a leaky surface: a boolean mask of
    packages (ids >= 2) whose values away from the surface get the wrong
    sign, and a mask of background cells whose far-package choice (inside /
    outside) is swapped where the cell is far."""
    st = Stream(seed)
    pk = st.uniform53(int(P)) < frac_pkg
    pk[:2] = False
    cells = st.uniform53(int(n_cells)) < frac_cell
    return pk, cells


def box_particles(n, lo, hi, seed=0):
    """n points uniform in the axis-aligned box [lo, hi)."""
    st = Stream(seed)
    u = st.uniform53(3 * n).reshape(3, n)
    return tuple(np.ascontiguousarray(lo[a] + u[a] * (hi[a] - lo[a]), dtype=np.float32)
                 for a in range(3))


# ----------------------------------------------------------------------------
# Random bodies (batched workloads)
# ----------------------------------------------------------------------------
def shape_area(s: Shape) -> float:
    """Closed-form surface area of a shape (used only to pick a spacing)."""
    if s.kind == SPHERE:
        return 4.0 * math.pi * s.p[0] ** 2
    if s.kind == TORUS:
        return 4.0 * math.pi ** 2 * s.p[0] * s.p[1]
    if s.kind == ROUNDED_BOX:
        a, b, c, r = (s.p[0] - s.p[3], s.p[1] - s.p[3], s.p[2] - s.p[3], s.p[3])
        return 8 * (a * b + b * c + a * c) + 4 * math.pi * r * (a + b + c) + 4 * math.pi * r * r
    raise ValueError("area not defined for kind %d" % s.kind)


def bounding_radius(s: Shape) -> float:
    if s.kind == SPHERE:
        return s.p[0]
    if s.kind == TORUS:
        return s.p[0] + s.p[1]
    if s.kind == ROUNDED_BOX:
        return math.sqrt(s.p[0] ** 2 + s.p[1] ** 2 + s.p[2] ** 2)
    raise ValueError("bounding radius not defined for kind %d" % s.kind)


def random_bodies(n, seed=1, p_lo=1e2, p_hi=1e5, kinds=(SPHERE, TORUS, ROUNDED_BOX),
                  pkg_per_area=4.6, margin_cells=4):
    """n random bodies, each with its own grid.

    Body k: kind uniform over ``kinds``; size r ~ U[0.1, 1]; uniform random
    rotation; a target package count log-uniform in [p_lo, p_hi] fixes the
    coarse cell lc = sqrt(pkg_per_area * area / target) and h = lc / 4.  The
    domain is a cube around the body with ``margin_cells`` coarse cells beyond
    its bounding sphere.  Returns a list of (Shape, GridSpec, target).
    """
    st = Stream(seed)
    out = []
    for _ in range(n):
        kind = kinds[int(st.uniform53(1)[0] * len(kinds)) % len(kinds)]
        r = 0.1 + 0.9 * st.uniform53(1)[0]
        rot = random_rotation(st)
        target = math.exp(math.log(p_lo) + st.uniform53(1)[0] * (math.log(p_hi) - math.log(p_lo)))
        if kind == SPHERE:
            s = sphere(r, rot=rot)
        elif kind == TORUS:
            s = torus(r, r / 3.0, rot=rot)
        else:
            s = rounded_box((r, 0.75 * r, 0.5 * r), 0.1 * r, rot=rot)
        lc = math.sqrt(pkg_per_area * shape_area(s) / target)
        h = lc / 4.0
        half = bounding_radius(s) + margin_cells * lc
        m = int(math.ceil(2.0 * half / lc))
        lo = tuple(-0.5 * m * lc for _ in range(3))
        out.append((s, GridSpec(lo, (m, m, m), h), target))
    return out


# ----------------------------------------------------------------------------
# Surrogate network initialisation
# ----------------------------------------------------------------------------
MLP_SHAPES = ((64, 27), (64,), (64, 64), (64,), (4, 64), (4,))


def mlp_init_params(seed=4):
    """Flat float32 parameter vector W1[64][27], b1, W2[64][64], b2, W3[4][64],
    b3 with every entry uniform in [-1/sqrt(fan_in), 1/sqrt(fan_in)),
    fan_in = 27, 27, 64, 64, 64, 64 (the layer's inputs)."""
    st = Stream(seed)
    fan = (27, 27, 64, 64, 64, 64)
    out = []
    for shape, f in zip(MLP_SHAPES, fan):
        n = int(np.prod(shape))
        a = 1.0 / math.sqrt(f)
        out.append((2.0 * st.uniform53(n) - 1.0) * a)
    return np.concatenate(out).astype(np.float32)
