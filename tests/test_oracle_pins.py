"""Pins of the FP64 oracle against things other than itself.

Each test fixes one part of the oracle by mathematics that does not go through
its code: closed-form distances, textbook constants of the Wendland kernel,
symmetry of the smoothed Heaviside, a library dilation for the band tagging,
a dense-array twin for the package tables and the index shift, exact fixed
points and closed-form single steps of the reinitialisation, and linear
reproduction of the trilinear probe.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.integrate
import scipy.ndimage

import oracle
import sg_inputs as si
from tests import dense_twin as dt


def tiny_sphere(h=0.0625, radius=0.55, n=8, centre=(0.03, -0.02, 0.05)):
    lc = 4 * h
    spec = si.GridSpec((-0.5 * n * lc,) * 3, (n, n, n), h)
    return si.sphere(radius, centre), spec


# ----------------------------------------------------------------------------
# Signed distance functions
# ----------------------------------------------------------------------------
def exact_lattice(v, lo, h):
    """Fine lattice index and weight of float32 coordinates v, from the
    definition u = (x - lo)/h - 1/2, i0 = floor(u), t = u - i0 evaluated in
    exact rational arithmetic (the binary values of v, lo and h)."""
    i0 = np.empty(len(v), np.int64)
    t = np.empty(len(v))
    Lo, H = Fraction(float(lo)), Fraction(float(h))
    for q, x in enumerate(np.asarray(v, np.float32)):
        u = (Fraction(float(x)) - Lo) / H - Fraction(1, 2)
        f = math.floor(u)
        i0[q] = f
        t[q] = float(u - f)
    return i0, t


def test_sdf_sphere_closed_form():
    s = si.sphere(0.7, centre=(0.1, 0.2, -0.3))
    d = oracle.sdf(s, [0.1, 1.1, 0.1], [0.2, 0.2, 0.2 + 0.7], [-0.3, -0.3, -0.3])
    assert np.allclose(d, [-0.7, 1.0 - 0.7, 0.0], atol=1e-15)


def test_sdf_plane_rotated():
    n = np.array([1.0, 2.0, -0.5])
    n /= np.linalg.norm(n)
    s = si.plane(n, point=(0.1, 0.0, 0.2))
    rng = np.random.default_rng(3)
    t = rng.uniform(-1, 1, 50)
    base = rng.uniform(-1, 1, (50, 3))
    base -= (base - np.array([0.1, 0.0, 0.2])) @ n[:, None] * n[None, :]  # project onto plane
    pts = base + t[:, None] * n[None, :]
    assert np.allclose(oracle.sdf(s, pts[:, 0], pts[:, 1], pts[:, 2]), t, atol=1e-14)


def test_sdf_torus_closed_form():
    R, r = 0.6, 0.2
    s = si.torus(R, r)
    # on the axis: distance to the core circle is sqrt(R^2 + z^2)
    z = np.array([0.0, 0.3, -0.7])
    assert np.allclose(oracle.sdf(s, 0 * z, 0 * z, z), np.sqrt(R * R + z * z) - r, atol=1e-15)
    # in the equatorial plane at angle u, radial distance rho from the axis
    u = np.linspace(0, 2 * np.pi, 7)
    rho = np.array([0.1, 0.4, 0.6, 0.8, 0.85, 1.2, 2.0])
    assert np.allclose(oracle.sdf(s, rho * np.cos(u), rho * np.sin(u), 0 * u), np.abs(rho - R) - r, atol=1e-15)


def test_sdf_rounded_box_closed_form():
    a, b, c, rr = 0.5, 0.3, 0.2, 0.05
    s = si.rounded_box((a, b, c), rr)
    # along the axes the distance is to the flat faces
    assert np.allclose(oracle.sdf(s, [a + 0.1, 0, 0], [0, b + 0.2, 0], [0, 0, -c - 0.3]), [0.1, 0.2, 0.3], atol=1e-15)
    # beyond a corner, the distance is to the corner sphere of radius rr
    p = np.array([a - rr, b - rr, c - rr]) + np.array([0.3, 0.4, 1.2])
    assert np.isclose(oracle.sdf(s, [p[0]], [p[1]], [p[2]])[0], 1.3 - rr, atol=1e-14)
    # at the centre: minus the smallest half extent
    assert np.isclose(oracle.sdf(s, [0], [0], [0])[0], -c, atol=1e-15)


def _brute_prism_distance(tri, z0, z1, pts, m=160):
    """Distance to the prism surface by dense sampling of its five faces."""
    T = np.asarray(tri)
    samples = []
    uu, vv = np.meshgrid(np.linspace(0, 1, m), np.linspace(0, 1, m))
    uu, vv = uu.ravel(), vv.ravel()
    keep = uu + vv <= 1.0
    cap = T[0] + uu[keep, None] * (T[1] - T[0]) + vv[keep, None] * (T[2] - T[0])
    for zc in (z0, z1):
        samples.append(np.column_stack([cap, np.full(len(cap), zc)]))
    for i in range(3):
        a, b = T[i], T[(i + 1) % 3]
        xy = a + uu[:, None] * (b - a)
        samples.append(np.column_stack([xy, z0 + vv * (z1 - z0)]))
    S = np.concatenate(samples)
    d = np.sqrt(((pts[:, None, :] - S[None, :, :]) ** 2).sum(-1)).min(1)
    return d


def _inside_prism(tri, z0, z1, pts):
    """Barycentric point-in-triangle test and slab test."""
    T = np.asarray(tri)
    v0, v1 = T[1] - T[0], T[2] - T[0]
    w = pts[:, :2] - T[0]
    den = v0[0] * v1[1] - v1[0] * v0[1]
    l1 = (w[:, 0] * v1[1] - v1[0] * w[:, 1]) / den
    l2 = (v0[0] * w[:, 1] - w[:, 0] * v0[1]) / den
    return (l1 > 0) & (l2 > 0) & (l1 + l2 < 1) & (pts[:, 2] > z0) & (pts[:, 2] < z1)


def test_sdf_prism_brute_force():
    tri, z0, z1 = si.PRISM_TRIANGLE, 0.0, 1.0
    s = si.prism(tri, z0, z1)
    rng = np.random.default_rng(7)
    pts = rng.uniform([-0.3, -0.3, -0.3], [1.3, 1.1, 1.3], (300, 3))
    d = oracle.sdf(s, pts[:, 0], pts[:, 1], pts[:, 2])
    ref = _brute_prism_distance(tri, z0, z1, pts)
    inside = _inside_prism(tri, z0, z1, pts)
    assert np.all((d < 0) == inside)
    # the sampled surface spacing is ~1/160: brute force overestimates by at most ~0.006
    assert np.all(np.abs(np.abs(d) - ref) < 7e-3)
    assert np.all(np.abs(d) <= ref + 1e-12)


def test_sdf_rotation_consistent():
    rot = si.random_rotation(si.Stream(11))
    R = np.asarray(rot).reshape(3, 3)
    s0 = si.torus(0.5, 0.15)
    s1 = si.torus(0.5, 0.15, centre=(0.2, -0.1, 0.3), rot=rot)
    rng = np.random.default_rng(5)
    q = rng.uniform(-1, 1, (40, 3))
    x = q @ R.T + np.array([0.2, -0.1, 0.3])
    assert np.allclose(oracle.sdf(s1, x[:, 0], x[:, 1], x[:, 2]), oracle.sdf(s0, q[:, 0], q[:, 1], q[:, 2]),
                       atol=1e-14)


@pytest.mark.parametrize("shape", [si.torus(0.5, 0.2), si.rounded_box((0.4, 0.3, 0.2), 0.05),
                                   si.prism(si.PRISM_TRIANGLE, 0.0, 1.0)])
def test_sdf_eikonal(shape):
    """|grad d| = 1 almost everywhere (finite differences away from kinks)."""
    rng = np.random.default_rng(2)
    p = rng.uniform(-0.6, 1.1, (400, 3))
    e = 1e-6
    g = np.stack([(oracle.sdf(shape, *(p + e * np.eye(3)[a]).T) - oracle.sdf(shape, *(p - e * np.eye(3)[a]).T))
                  / (2 * e) for a in range(3)], 1)
    n = np.linalg.norm(g, axis=1)
    assert np.mean(np.abs(n - 1) < 1e-5) > 0.9  # medial-axis points are the exception
    assert np.all(n < 1 + 1e-5)


# ----------------------------------------------------------------------------
# Tagging, ids and tables
# ----------------------------------------------------------------------------
def _brute_tags(spec, shape):
    nx, ny, nz = spec.dims
    h = spec.h
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    x = spec.lo[0] + (4.0 * I + 2.0) * h
    y = spec.lo[1] + (4.0 * J + 2.0) * h
    z = spec.lo[2] + (4.0 * K + 2.0) * h
    d = oracle.sdf(shape, x.ravel(), y.ravel(), z.ravel()).reshape(nz, ny, nx)
    T = 4 * h * (1 - 2.0 ** -10)
    core = np.abs(d) < T
    dil = scipy.ndimage.binary_dilation(core, structure=np.ones((3, 3, 3), bool))
    inner = dil & ~core
    active = (core | inner).ravel()
    ids = np.where(active, 2 + np.cumsum(active) - 1, np.where(d.ravel() < 0, 0, 1))
    return ids.astype(np.int32), core.ravel(), inner.ravel()


@pytest.mark.parametrize("case", ["sphere", "torus", "box"])
def test_tagging_brute_force(case):
    if case == "sphere":
        shape, spec = tiny_sphere()
    elif case == "torus":
        shape = si.torus(0.45, 0.15, rot=si.random_rotation(si.Stream(4)))
        spec = si.GridSpec((-0.8, -0.8, -0.8), (20, 20, 20), 0.02)
    else:
        shape = si.rounded_box((0.5, 0.35, 0.25), 0.06, rot=si.random_rotation(si.Stream(9)))
        spec = si.GridSpec((-0.9, -0.9, -0.9), (18, 18, 18), 0.025)
    cell_pkg, cell_type, P, ties = oracle.tag(spec, shape)
    ids, core, inner = _brute_tags(spec, shape)
    assert ties == 0
    assert np.array_equal(cell_pkg, ids)
    assert np.array_equal(cell_type == 2, core)
    assert np.array_equal(cell_type == 3, inner)
    assert P == 2 + int((core | inner).sum())


def test_tables_invariants():
    shape, spec = si.sphere_small()
    G = oracle.build_grid(spec, shape)
    P, nbr, pc, pt, cp = G.P, G.nbr, G.pkg_cell, G.pkg_type, G.cell_pkg
    nx, ny, nz = spec.dims
    assert np.all(nbr[0] == 0) and np.all(nbr[1] == 1)
    assert list(pt[:2]) == [0, 1] and list(pc[:2]) == [-1, -1]
    assert np.array_equal(nbr[2:, 13], np.arange(2, P))
    assert np.array_equal(cp[pc[2:]], np.arange(2, P))
    assert np.all(np.diff(pc[2:]) > 0)  # ids increase with cell index
    core = np.where(pt == 2)[0]
    assert np.all(nbr[core] >= 2)  # every neighbour of a core cell is active
    # neighbour entries point at the cell with the right offset
    for p in (2, P // 2, P - 1):
        c = pc[p]
        I, J, K = c % nx, (c // nx) % ny, c // (nx * ny)
        for n in range(27):
            di, dj, dk = n % 3 - 1, (n // 3) % 3 - 1, n // 9 - 1
            a, b, e = I + di, J + dj, K + dk
            inside = 0 <= a < nx and 0 <= b < ny and 0 <= e < nz
            assert nbr[p, n] == (cp[a + nx * (b + ny * e)] if inside else 1)


def test_sphere_small_counts():
    shape, spec = si.sphere_small()
    cell_pkg, cell_type, P, ties = oracle.tag(spec, shape)
    ids, core, inner = _brute_tags(spec, shape)
    assert np.array_equal(cell_pkg, ids)
    assert (P, int(core.sum()), int(inner.sum()), ties) == (1634, 638, 994, 0)


# ----------------------------------------------------------------------------
# Dense twin: tables + index shift, bit for bit
# ----------------------------------------------------------------------------
@pytest.fixture(scope="module")
def tiny():
    shape, spec = tiny_sphere()
    G = oracle.build_grid(spec, shape)
    rng = np.random.default_rng(0)
    # perturb phi so that no stencil sees a symmetric field
    G.phi[2:] += rng.normal(0, 0.01, G.phi[2:].shape)
    G.F = oracle.far_value(spec)
    G.D = dt.to_dense(spec, G.cell_pkg, G.cell_type, G.phi, G.F)
    return G


def _act(G):
    return G.pkg_type >= 2


def test_dense_twin_gradient(tiny):
    G = tiny
    ref = [dt.from_dense(G.spec, G.cell_pkg, G.cell_type, np.pad(g, dt.PAD), G.P)
           for g in dt.gradient(G.D, G.spec.h)]
    got = oracle.gradient(G.spec, G.nbr, G.phi)
    for a in range(3):
        assert np.array_equal(got[a][_act(G)], ref[a][_act(G)])
        assert np.all(got[a][:2] == 0)


def test_dense_twin_laplacian(tiny):
    G = tiny
    ref = dt.from_dense(G.spec, G.cell_pkg, G.cell_type, np.pad(dt.laplacian(G.D, G.spec.h), dt.PAD), G.P)
    got = oracle.laplacian(G.spec, G.nbr, G.phi)
    assert np.array_equal(got[_act(G)], ref[_act(G)])


def test_dense_twin_reinit_step(tiny):
    G = tiny
    h = G.spec.h
    s0 = oracle.reinit_s0(G.spec, G.phi)
    S0 = dt.to_dense(G.spec, G.cell_pkg, G.cell_type, s0, 1.0)
    new = dt.reinit_step(G.D, G.D, S0, h, 0.5 * h)
    ref = dt.from_dense(G.spec, G.cell_pkg, G.cell_type, np.pad(new, dt.PAD), G.P)
    got = oracle.reinit_step(G.spec, G.nbr, G.phi, s0, G.phi, 0.5 * h)
    assert np.array_equal(got[_act(G)], ref[_act(G)])
    assert np.array_equal(got[:2], G.phi[:2])


def test_dense_twin_kernel_integrals(tiny):
    G = tiny
    ref = [dt.from_dense(G.spec, G.cell_pkg, G.cell_type, np.pad(v, dt.PAD), G.P)
           for v in dt.kernel_integrals(G.D, G.spec.h)]
    got = oracle.kernel_integrals(G.spec, G.nbr, G.phi)
    for a in range(4):
        # numpy and libm sines may differ in the last bit; sums of 27 taps
        assert np.max(np.abs(got[a][_act(G)] - ref[a][_act(G)])) < 1e-14
    assert np.all(got[0][0] == 1) and np.all(got[0][1] == 0)
    for a in range(1, 4):
        assert np.all(got[a][:2] == 0)


def test_dense_twin_probe(tiny):
    """Trilinear probe on the dense twin: corners are plain array lookups.

    A particle whose home cell is far reads the far package for all eight
    corners (far packages are their own neighbours), so the reference takes
    the far constant there."""
    G = tiny
    spec = G.spec
    h = spec.h
    fields = [G.phi, *oracle.gradient(spec, G.nbr, G.phi), *oracle.kernel_integrals(spec, G.nbr, G.phi)]
    x, y, z = si.box_particles(3000, spec.lo, spec.hi(), seed=5)
    got = oracle.probe(spec, G.cell_pkg, G.nbr, fields, x, y, z)
    nx, ny, nz = spec.dims
    i0, t = [], []
    for a, v in enumerate((x, y, z)):
        ia, ta = exact_lattice(v, spec.lo[a], h)
        i0.append(ia)
        t.append(ta)
    I = [v // 4 for v in i0]
    inside = (I[0] >= 0) & (I[1] >= 0) & (I[2] >= 0) & (I[0] < nx) & (I[1] < ny) & (I[2] < nz)
    cidx = np.clip(I[0], 0, nx - 1) + nx * (np.clip(I[1], 0, ny - 1) + ny * np.clip(I[2], 0, nz - 1))
    home_type = np.where(inside, G.cell_type[cidx], 1)
    for f_i, f in enumerate(fields):
        f_in, f_out = f[0][0], f[1][0]
        D = dt.to_dense(spec, G.cell_pkg, G.cell_type, f, f_out, far_in=f_in)
        acc = np.zeros(len(x))
        for c in range(8):
            a0, a1, a2 = c & 1, (c >> 1) & 1, (c >> 2) & 1
            w = (t[0] if a0 else 1 - t[0]) * (t[1] if a1 else 1 - t[1]) * (t[2] if a2 else 1 - t[2])
            acc = acc + w * D[i0[2] + a2 + dt.PAD, i0[1] + a1 + dt.PAD, i0[0] + a0 + dt.PAD]
        ref = np.where(home_type >= 2, acc, np.where(home_type == 0, f_in, f_out))
        if f_i in (1, 2, 3):
            continue  # gradients are normalised below
        assert np.max(np.abs(got[f_i] - ref)) < 1e-13, f_i
    g = []
    for f_i in (1, 2, 3):
        D = dt.to_dense(spec, G.cell_pkg, G.cell_type, fields[f_i], 0.0, far_in=0.0)
        acc = np.zeros(len(x))
        for c in range(8):
            a0, a1, a2 = c & 1, (c >> 1) & 1, (c >> 2) & 1
            w = (t[0] if a0 else 1 - t[0]) * (t[1] if a1 else 1 - t[1]) * (t[2] if a2 else 1 - t[2])
            acc = acc + w * D[i0[2] + a2 + dt.PAD, i0[1] + a1 + dt.PAD, i0[0] + a0 + dt.PAD]
        g.append(np.where(home_type >= 2, acc, 0.0))
    gn = np.sqrt(g[0] ** 2 + g[1] ** 2 + g[2] ** 2)
    for a in range(3):
        ref = np.where(gn > 0, g[a] / np.where(gn > 0, gn, 1), 0.0)
        assert np.max(np.abs(got[1 + a] - ref)) < 1e-12


# ----------------------------------------------------------------------------
# Gradient
# ----------------------------------------------------------------------------
def _interior_packages(G):
    """Active packages whose 26 neighbours are all active."""
    return np.where((G.pkg_type >= 2) & np.all(G.nbr >= 2, axis=1))[0]


def test_gradient_plane_exact():
    n = np.array([0.3, -0.5, 0.8])
    n /= np.linalg.norm(n)
    shape = si.plane(n, point=(0.01, 0.02, -0.03))
    spec = si.GridSpec((-0.5, -0.5, -0.5), (10, 10, 10), 0.025)
    G = oracle.build_grid(spec, shape)
    g = oracle.gradient(spec, G.nbr, G.phi)
    ip = _interior_packages(G)
    assert len(ip) > 20
    for a in range(3):
        assert np.max(np.abs(g[a][ip] - n[a])) < 1e-12


def test_gradient_sphere_second_order():
    errs = []
    for h in (0.04, 0.02):
        spec = si.GridSpec((-1.6, -1.6, -1.6), (int(round(3.2 / (4 * h))),) * 3, h)
        G = oracle.build_grid(spec, si.sphere(1.0))
        g = oracle.gradient(spec, G.nbr, G.phi)
        core = G.pkg_type == 2
        nrm = np.sqrt(g[0] ** 2 + g[1] ** 2 + g[2] ** 2)[core]
        errs.append(np.max(np.abs(nrm - 1)))
    # central differences of |x| - 1 have error ~ h^2 / R^2
    assert errs[0] < 0.5 * 0.04 ** 2 / 0.8 ** 2
    assert 3.0 < errs[0] / errs[1] < 6.0


# ----------------------------------------------------------------------------
# Reinitialisation
# ----------------------------------------------------------------------------
def _fine_coords(G):
    """Fine lattice indices (i, j, k) of every data point, shape (P, 64)."""
    nx, ny, _ = G.spec.dims
    pc = G.pkg_cell.astype(np.int64)
    I, J, K = pc % nx, (pc // nx) % ny, pc // (nx * ny)
    d = np.arange(64)
    return (4 * I[:, None] + d % 4, 4 * J[:, None] + (d // 4) % 4, 4 * K[:, None] + d // 16)


def test_reinit_plane_fixed_point():
    """A plane is a fixed point of the Godunov update.  A plane meets the
    domain boundary, where neighbours outside read +F; Jacobi sweeps carry
    that one fine cell per iteration, so only points deeper than the
    iteration count are checked."""
    n = np.array([0.2, 0.9, -0.4])
    n /= np.linalg.norm(n)
    shape = si.plane(n, point=(0.013, -0.02, 0.031))
    spec = si.GridSpec((-0.6, -0.6, -0.6), (12, 12, 12), 0.025)
    G = oracle.build_grid(spec, shape)
    iters = 8
    phi = oracle.reinit(spec, G.nbr, G.phi, iters, 0.5)
    fi = _fine_coords(G)
    deep = np.ones(G.phi.shape, bool)
    for a in range(3):
        deep &= (fi[a] > iters) & (fi[a] < 4 * spec.dims[a] - 1 - iters)
    sel = deep & (G.pkg_type[:, None] >= 2)
    sel[:2] = False
    assert sel.sum() > 5000
    assert np.max(np.abs(phi[sel] - G.phi[sel])) < 1e-13
    assert np.array_equal(phi[:2], G.phi[:2])


def test_reinit_constant_field_closed_form():
    """On a flat field a = b = 0, so G = 0 and phi moves by +dt S0 exactly."""
    shape, spec = tiny_sphere()
    G = oracle.build_grid(spec, shape)
    h = spec.h
    for c in (0.01, -0.02):
        phi = G.phi.copy()
        phi[2:] = c
        s0 = oracle.reinit_s0(spec, phi)
        out = oracle.reinit_step(spec, G.nbr, phi, s0, phi, 0.5 * h)
        ip = _interior_packages(G)
        expect = c - 0.5 * h * (c / math.sqrt(c * c + h * h)) * (0.0 - 1.0)
        assert np.all(out[ip] == expect)


def test_reinit_linear_slope_closed_form():
    """phi = s * (plane distance): G = s^2, so phi moves by -dt S0 (|s| - 1)."""
    n = np.array([1.0, 0.0, 0.0])
    shape = si.plane(n, point=(0.0123, 0.0, 0.0))
    spec = si.GridSpec((-0.5, -0.5, -0.5), (10, 10, 10), 0.025)
    G = oracle.build_grid(spec, shape)
    h = spec.h
    for s in (2.0, 0.5):
        phi = G.phi.copy()
        phi[2:] *= s
        s0 = oracle.reinit_s0(spec, phi)
        out = oracle.reinit_step(spec, G.nbr, phi, s0, phi, 0.5 * h)
        ip = _interior_packages(G)
        expect = phi[ip] - 0.5 * h * s0[ip] * (s - 1.0)
        assert np.max(np.abs(out[ip] - expect)) < 1e-15


def test_reinit_godunov_branches():
    """Kinks: a positive minimum rises by dt S0 (G = 0); a positive maximum
    (shock) takes the steeper side; for negative phi the roles swap."""
    shape = si.plane((1.0, 0.0, 0.0), point=(0.0, 0.0, 0.0))
    spec = si.GridSpec((-0.5, -0.5, -0.5), (10, 10, 10), 0.025)
    G = oracle.build_grid(spec, shape)
    h = spec.h
    ip = _interior_packages(G)
    # build phi = c + alpha |x - x0| style kinks along x on the fine lattice
    nx = spec.dims[0]
    pc = G.pkg_cell
    I = (pc % nx).astype(np.int64)
    ii = np.tile(np.arange(4), 16)
    fine_x = 4 * I[:, None] + ii[None, :]
    x0 = 20
    for c, slope_l, slope_r, G_expect in ((0.05, -1.0, 1.0, 0.0),   # positive minimum
                                          (0.05, 2.0, -3.0, 9.0),   # positive maximum: steeper side
                                          (-0.05, 2.0, -3.0, 0.0),  # negative maximum
                                          (-0.05, -1.0, 2.0, 4.0)):  # negative minimum: steeper side
        dx = (fine_x - x0).astype(np.float64) * h
        phi = np.where(dx < 0, c + slope_l * dx, c + slope_r * dx)
        phi[:2] = G.phi[:2]
        s0 = oracle.reinit_s0(spec, phi)
        out = oracle.reinit_step(spec, G.nbr, phi, s0, phi, 0.5 * h)
        at = (fine_x == x0)
        sel = np.zeros_like(at)
        sel[ip] = at[ip]
        expect = c - 0.5 * h * s0[sel] * (math.sqrt(G_expect) - 1.0)
        assert np.max(np.abs(out[sel] - expect)) < 1e-15


def test_reinit_distorted_sphere_converges():
    shape, spec = si.sphere_small()
    G = oracle.build_grid(spec, shape)
    h = spec.h
    nx, ny, nz = spec.dims
    pc = G.pkg_cell[2:]
    I, J, K = pc % nx, (pc // nx) % ny, pc // (nx * ny)
    d = np.arange(64)
    i, j, k = d % 4, (d // 4) % 4, d // 16
    x = spec.lo[0] + (4 * I[:, None] + i[None, :] + 0.5) * h
    y = spec.lo[1] + (4 * J[:, None] + j[None, :] + 0.5) * h
    z = spec.lo[2] + (4 * K[:, None] + k[None, :] + 0.5) * h
    phi = G.phi.copy()
    phi[2:] = G.phi[2:] * (0.5 + x * x + y * y + z * z)
    out = oracle.reinit(spec, G.nbr, phi, 80, 0.5)
    g = oracle.gradient(spec, G.nbr, out)
    core = G.pkg_type == 2
    nrm = np.sqrt(g[0] ** 2 + g[1] ** 2 + g[2] ** 2)[core]
    assert np.max(np.abs(nrm - 1.0)) < 0.05
    # the zero crossing stays put: compare with the exact distance near the surface
    near = core[:, None] & (np.abs(G.phi) < 0.5 * h)
    assert np.max(np.abs(out[near] - G.phi[near])) < 0.5 * h


# ----------------------------------------------------------------------------
# Kernel and Heaviside
# ----------------------------------------------------------------------------
def test_wendland_textbook_normalisation():
    """Wendland C2 in 3-D: int w(|r|) d^3r over support 2 equals 16 pi / 21."""
    val, _ = scipy.integrate.quad(lambda q: oracle.wendland(q) * 4 * math.pi * q * q, 0, 2)
    assert abs(val - 16 * math.pi / 21) < 1e-12


def test_wendland_derivative_and_support():
    for q in (0.1, 0.7, 1.0, 1.5, 1.9):
        e = 1e-6
        fd = (oracle.wendland(q + e) - oracle.wendland(q - e)) / (2 * e)
        assert abs(fd - oracle.wendland_dq(q)) < 1e-8
    assert oracle.wendland(0) == 1.0 and oracle.wendland(2) == 0 and oracle.wendland_dq(2) == 0
    assert oracle.wendland(2.5) == 0 and oracle.wendland(1.999999) > 0


def test_heaviside_symmetry():
    eps = 0.3
    zs = np.linspace(-0.5, 0.5, 101)
    for z in zs:
        assert abs(oracle.heaviside(z, eps) + oracle.heaviside(-z, eps) - 1) < 1e-15
    assert oracle.heaviside(0.0, eps) == 0.5
    assert oracle.heaviside(-0.31, eps) == 0 and oracle.heaviside(0.31, eps) == 1
    assert abs(oracle.heaviside(eps, eps) - 1) < 1e-15 and abs(oracle.heaviside(-eps, eps)) < 1e-15
    e = 1e-7
    assert abs((oracle.heaviside(e, eps) - oracle.heaviside(-e, eps)) / (2 * e) - 1 / eps) < 1e-6
    val, _ = scipy.integrate.quad(lambda z: oracle.heaviside(z, eps), -eps, eps)
    assert abs(val - eps) < 1e-12


def _plane_grid(offset_layers=0.0):
    """Plane z = z0 on a dyadic lattice; z0 = data layer + offset_layers * h."""
    h = 2.0 ** -5
    spec = si.GridSpec((-0.5, -0.5, -0.5), (8, 8, 8), h)
    z0 = spec.lo[2] + (15 + 0.5) * h + offset_layers * h
    shape = si.plane((0.0, 0.0, 1.0), point=(0.0, 0.0, z0))
    return shape, spec, z0


def _plane_reduction(delta_over_h):
    """1-D reduction of the 27-tap sums for phi = delta + s_z h: group taps by s_z."""
    A = {m: 0.0 for m in (-1, 0, 1)}
    B = {m: 0.0 for m in (-1, 0, 1)}
    for sx in (-1, 0, 1):
        for sy in (-1, 0, 1):
            for m in (-1, 0, 1):
                q = math.sqrt(sx * sx + sy * sy + m * m)
                t = 1 - q / 2
                A[m] += t ** 4 * (1 + 2 * q)
                if q > 0:
                    B[m] += -5 * q * t ** 3 * (-m) / q
    den = sum(A.values())

    def H(z):
        return 0.0 if z < -1 else (1.0 if z > 1 else 0.5 * (1 + z + math.sin(math.pi * z) / math.pi))

    W = sum(A[m] * H(-(delta_over_h + m)) for m in A) / den
    Gz = sum(B[m] * H(-(delta_over_h + m)) for m in B) / den
    return W, Gz, A, den


@pytest.mark.parametrize("offset", [0.0, -0.5, -1.0, 0.25])
def test_integrals_plane_closed_form(offset):
    shape, spec, z0 = _plane_grid(offset)
    G = oracle.build_grid(spec, shape)
    W, Gx, Gy, Gz = oracle.kernel_integrals(spec, G.nbr, G.phi)
    ip = _interior_packages(G)
    h = spec.h
    nz = spec.dims[2]
    K = G.pkg_cell[ip] // (spec.dims[0] * spec.dims[1])
    kk = np.arange(64) // 16
    zc = spec.lo[2] + (4 * K[:, None] + kk[None, :] + 0.5) * h
    delta = (zc - z0) / h
    for dv in np.unique(np.round(delta, 12)):
        if abs(dv) > 3:
            continue
        sel = np.abs(delta - dv) < 1e-9
        Wr, Gr, _, _ = _plane_reduction(dv)
        assert np.max(np.abs(W[ip][sel] - Wr)) < 1e-14
        assert np.max(np.abs(Gz[ip][sel] - Gr)) < 1e-14
        assert np.max(np.abs(Gx[ip][sel])) < 1e-15 and np.max(np.abs(Gy[ip][sel])) < 1e-15


def test_integrals_plane_half_and_tap_weights():
    shape, spec, z0 = _plane_grid(0.0)
    G = oracle.build_grid(spec, shape)
    W, Gx, Gy, Gz = oracle.kernel_integrals(spec, G.nbr, G.phi)
    on = (np.abs(G.phi) == 0.0) & (G.pkg_type[:, None] >= 2)
    ip = np.zeros(G.P, bool)
    ip[_interior_packages(G)] = True
    on &= ip[:, None]
    assert on.sum() > 0
    assert np.max(np.abs(W[on] - 0.5)) < 1e-15  # symmetry: half the kernel mass
    # the normalised tap weights of the four distance classes
    den = oracle.wendland(0) + 6 * oracle.wendland(1) + 12 * oracle.wendland(math.sqrt(2)) + \
        8 * oracle.wendland(math.sqrt(3))
    assert abs(oracle.wendland(0) / den - 0.4041055771) < 1e-10
    assert abs(oracle.wendland(1) / den - 0.0757697957) < 1e-10
    assert abs(oracle.wendland(math.sqrt(2)) / den - 0.0113855102) < 1e-10
    assert abs(oracle.wendland(math.sqrt(3)) / den - 0.0005811908) < 1e-10
    assert np.max(np.abs(Gz[on] + 0.475074612)) < 1e-9


def test_integrals_deep_inside_outside():
    shape, spec = si.sphere_small()
    G = oracle.build_grid(spec, shape)
    W, Gx, Gy, Gz = oracle.kernel_integrals(spec, G.nbr, G.phi)
    h = spec.h
    act = G.pkg_type >= 2
    ip = np.zeros(G.P, bool)
    ip[_interior_packages(G)] = True
    # every tap (|s| <= sqrt 3) beyond eps = h from the surface
    deep_in = (G.phi < -2.8 * h) & ip[:, None]
    deep_out = (G.phi > 2.8 * h) & ip[:, None]
    assert deep_in.sum() > 100 and deep_out.sum() > 100
    assert np.all(W[deep_in] == 1.0) and np.all(W[deep_out] == 0.0)
    for g in (Gx, Gy, Gz):
        # opposite taps cancel up to the rounding of the running sum
        assert np.max(np.abs(g[deep_in])) < 1e-15 and np.all(g[deep_out] == 0.0)
    # far packages carry the limits
    assert np.all(W[0] == 1.0) and np.all(W[1] == 0.0)
    assert np.all((W[act] >= 0) & (W[act] <= 1))


# ----------------------------------------------------------------------------
# Probe and Morton order
# ----------------------------------------------------------------------------
def test_probe_reproduces_linear_field():
    n = np.array([0.6, -0.3, 0.74])
    n /= np.linalg.norm(n)
    p0 = np.array([0.011, -0.017, 0.023])
    shape = si.plane(n, point=tuple(p0))
    spec = si.GridSpec((-0.5, -0.5, -0.5), (10, 10, 10), 0.025)
    G = oracle.build_grid(spec, shape)
    fields = [G.phi, *oracle.gradient(spec, G.nbr, G.phi), *oracle.kernel_integrals(spec, G.nbr, G.phi)]
    x, y, z = si.box_particles(4000, (-0.15,) * 3, (0.15,) * 3, seed=3)
    out = oracle.probe(spec, G.cell_pkg, G.nbr, fields, x, y, z)
    # interpolation reproduces a linear field at the particle's own position
    pts = np.stack([np.asarray(v, np.float32).astype(np.float64) for v in (x, y, z)], 1)
    exact = (pts - p0) @ n
    ok = np.abs(exact) < 4 * spec.h  # all eight corners in the interior of the band
    assert ok.sum() > 1000
    assert np.max(np.abs(out[0][ok] - exact[ok])) < 1e-13
    for a in range(3):
        assert np.max(np.abs(out[1 + a][ok] - n[a])) < 1e-12


def test_probe_quadratic_field_picks_the_enclosing_cell():
    """Trilinear interpolation of f = X^2 (X the data point's x coordinate)
    between the corners of the cell that encloses the particle overshoots by
    exactly h^2 t (1 - t), t in [0, 1); corners one cell off would extrapolate
    and undershoot.  So this pins the cell decision and the weight t against
    exact rational arithmetic, not against the oracle's own formula."""
    spec = si.GridSpec((-0.3, -0.3, -0.3), (6, 6, 6), 0.025)
    G = oracle.build_grid(spec, si.sphere(0.2, (0.0, 0.0, 0.0)))
    assert G.P == 2 + 6 ** 3  # every cell active: all corners below are data points
    X = spec.lo[0] + (_fine_coords(G)[0] + 0.5) * spec.h
    fx = X * X
    zero = np.zeros_like(fx)
    fields = [fx, zero, zero, zero, zero, zero, zero, zero]
    x, y, z = si.box_particles(3000, (-0.28,) * 3, (0.28,) * 3, seed=11)
    out = oracle.probe(spec, G.cell_pkg, G.nbr, fields, x, y, z)[0]
    i0, t = exact_lattice(x, spec.lo[0], spec.h)
    xs = np.asarray(x, np.float32).astype(np.float64)
    expect = xs * xs + spec.h ** 2 * t * (1.0 - t)
    assert oracle.lattice_ties(spec, x, y, z) == 0
    assert np.all((t >= 0) & (t < 1))
    assert np.max(np.abs(out - expect)) < 1e-12


def test_probe_at_data_points_and_far():
    shape, spec = si.sphere_small()
    G = oracle.build_grid(spec, shape)
    fields = [G.phi, *oracle.gradient(spec, G.nbr, G.phi), *oracle.kernel_integrals(spec, G.nbr, G.phi)]
    nx, ny, nz = spec.dims
    h = spec.h
    rng = np.random.default_rng(1)
    ps = rng.integers(2, G.P, 200)
    # in-package indices 1..3: a float32 rounding just below the data point
    # keeps the particle in the same (active) home package
    i, j, k = (rng.integers(1, 4, 200) for _ in range(3))
    ds = i + 4 * j + 16 * k
    c = G.pkg_cell[ps]
    I, J, K = c % nx, (c // nx) % ny, c // (nx * ny)
    x = (np.float32(spec.lo[0]) + (4 * I + i + np.float32(0.5)) * np.float32(h)).astype(np.float32)
    y = (np.float32(spec.lo[1]) + (4 * J + j + np.float32(0.5)) * np.float32(h)).astype(np.float32)
    z = (np.float32(spec.lo[2]) + (4 * K + k + np.float32(0.5)) * np.float32(h)).astype(np.float32)
    out = oracle.probe(spec, G.cell_pkg, G.nbr, fields, x, y, z)
    # float32 positions are within an ulp of the data points: values agree to O(ulp * |grad|)
    assert np.max(np.abs(out[0] - G.phi[ps, ds])) < 1e-5
    assert np.max(np.abs(out[4] - fields[4][ps, ds])) < 1e-3
    # far inside (origin) and far outside (a corner of the domain), and outside the domain
    F = oracle.far_value(spec)
    x2 = np.array([0.0, 1.45, 5.0], np.float32)
    o2 = oracle.probe(spec, G.cell_pkg, G.nbr, fields, x2, np.zeros(3, np.float32) + [0, 1.45, 0],
                      np.zeros(3, np.float32) + [0, 1.45, 0])
    # eight equal corners, weights summing to 1 up to rounding
    assert np.max(np.abs(o2[0] - np.array([-F, F, F]))) < 1e-14
    assert np.max(np.abs(o2[4] - np.array([1.0, 0.0, 0.0]))) < 1e-15
    for a in (1, 2, 3, 5, 6, 7):
        assert list(o2[a]) == [0.0, 0.0, 0.0]


def test_morton_keys_bit_loop():
    spec = si.GridSpec((-1.0, -1.0, -1.0), (50, 50, 50), 0.01)
    x, y, z = si.box_particles(300, (-1.2,) * 3, (1.2,) * 3, seed=8)
    keys = oracle.morton_keys(spec, x, y, z)
    for q in range(0, 300, 7):
        k = []
        for a, v in enumerate((x[q], y[q], z[q])):
            i0 = int(exact_lattice([v], spec.lo[a], spec.h)[0][0])
            k.append(min(max(i0 + 1, 0), 4 * spec.dims[a] + 1))
        ref = 0
        for b in range(21):
            for a in range(3):
                if (k[a] >> b) & 1:
                    ref += 2 ** (3 * b + a)
        assert int(keys[q]) == ref


def test_morton_order_stable():
    rng = np.random.default_rng(4)
    keys = rng.integers(0, 50, 5000).astype(np.uint64)  # many ties
    order = oracle.morton_order(keys)
    assert np.array_equal(order, np.argsort(keys, kind="stable"))


def test_sdf_shell_closed_form():
    """Shell between radii 0.3 and 0.31 about (0.5, 0.5, 0.5): distance to the
    nearer of the two spheres, negative between them."""
    s = si.shell(0.3, 0.31, (0.5, 0.5, 0.5))
    d = np.array([0.6, -1.0, 0.25])
    d /= np.linalg.norm(d)
    r = np.array([0.0, 0.1, 0.3, 0.302, 0.305, 0.309, 0.31, 0.5])
    pts = 0.5 + r[:, None] * d[None, :]
    got = oracle.sdf(s, pts[:, 0], pts[:, 1], pts[:, 2])
    expect = np.where(r < 0.305, 0.3 - r, r - 0.31)
    assert np.allclose(got, expect, atol=1e-15)
    # the thickest inside point is the mid radius, at minus half the thickness
    assert abs(got[4] + 0.005) < 1e-15


def test_sequential_update_is_plain_addition():
    phi = np.arange(5 * 64, dtype=np.float32).reshape(5, 64) * np.float32(0.001)
    out = oracle.sequential(phi, 1e-3)
    assert np.array_equal(out[:2], phi[:2])
    assert np.array_equal(out[2:], phi[2:] + np.float32(1e-3))
