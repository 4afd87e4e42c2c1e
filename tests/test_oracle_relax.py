"""Pins of the oracle's particle relaxation (each step: probe, then move by
-s h clip(phi/h, -1, 1) n, positions stored in float32).

On a plane the interpolated phi and the central-difference normal are exact,
so the signed distance of a particle follows the scalar recurrence
d <- d - s h clip(d/h, -1, 1) and its tangential position does not change;
a particle whose corners all lie in a far package sees n = 0 and stays put;
on a sphere particles converge radially onto the surface.
"""
import numpy as np

import oracle
import sg_inputs as si

F32_EPS = 2.0 ** -23


def _plane_setup():
    n = np.array([0.3, -0.5, 0.8])
    n /= np.linalg.norm(n)
    c = np.array([0.01, 0.02, -0.03])
    shape = si.plane(n, point=tuple(c))
    spec = si.GridSpec((-0.5, -0.5, -0.5), (10, 10, 10), 0.025)
    G = oracle.build_grid(spec, shape)
    g = oracle.gradient(spec, G.nbr, G.phi)
    zero = np.zeros_like(G.phi)
    fields = (G.phi, g[0], g[1], g[2], zero, zero, zero, zero)
    return n, c, spec, G, fields


def _plane_particles(n, c, d, seed):
    st = si.Stream(seed)
    u = 0.3 * (2.0 * st.uniform53(3 * d.size).reshape(-1, 3) - 1.0)
    u -= (u @ n)[:, None] * n[None, :]  # tangential offsets, |u| < 0.52
    p = c[None, :] + u + d[:, None] * n[None, :]
    p = p.astype(np.float32)
    return p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy()


def test_relax_plane_recurrence():
    n, c, spec, G, fields = _plane_setup()
    h = spec.h
    st = si.Stream(11)
    d0 = (2.0 * st.uniform53(3000) - 1.0) * 3.0 * h  # clipped and unclipped moves, both sides
    x, y, z = _plane_particles(n, c, d0, 12)
    P0 = np.stack([x, y, z], 1).astype(np.float64)
    d_start = (P0 - c[None, :]) @ n  # distances after rounding the start to float32
    K = 20
    (xk, yk, zk), out = oracle.relax(spec, G.cell_pkg, G.nbr, fields, x, y, z, K, 0.1)
    PK = np.stack([xk, yk, zk], 1).astype(np.float64)
    d = d_start.copy()
    for _ in range(K):
        d = d - 0.1 * h * np.clip(d / h, -1.0, 1.0)
    tol = K * F32_EPS * np.max(np.abs(P0))
    assert np.max(np.abs((PK - c[None, :]) @ n - d)) <= tol
    # the move is along n only
    dt = (PK - P0) - ((PK - P0) @ n)[:, None] * n[None, :]
    assert np.max(np.linalg.norm(dt, axis=1)) <= tol
    # the last step's probe: phi of the start of that step, n exact
    assert np.max(np.abs(out[1] - n[0])) < 1e-9
    assert np.max(np.abs(out[3] - n[2])) < 1e-9


def test_relax_far_particles_stay():
    n, c, spec, G, fields = _plane_setup()
    d0 = np.full(500, -0.36)  # beyond the band: the home cell and its corners are far-
    x, y, z = _plane_particles(n, c, d0, 13)
    inside = (np.abs(x) < 0.45) & (np.abs(y) < 0.45) & (np.abs(z) < 0.45)  # home cells in the domain
    x, y, z = x[inside], y[inside], z[inside]
    assert x.size > 100
    (xk, yk, zk), out = oracle.relax(spec, G.cell_pkg, G.nbr, fields, x, y, z, 5, 0.1)
    F = 16.0 * spec.h
    assert np.max(np.abs(out[0] + F)) <= 1e-12 * F  # weights sum to 1 up to rounding
    assert np.all(out[1] == 0.0) and np.all(out[2] == 0.0) and np.all(out[3] == 0.0)
    assert np.array_equal(xk, x) and np.array_equal(yk, y) and np.array_equal(zk, z)


def test_relax_sphere_converges_radially():
    h = 0.04
    spec = si.GridSpec((-1.6, -1.6, -1.6), (20, 20, 20), h)
    G = oracle.build_grid(spec, si.sphere(1.0))
    g = oracle.gradient(spec, G.nbr, G.phi)
    zero = np.zeros_like(G.phi)
    fields = (G.phi, g[0], g[1], g[2], zero, zero, zero, zero)
    st = si.Stream(14)
    z0 = 2.0 * st.uniform53(2000) - 1.0
    az = 2.0 * np.pi * st.uniform53(2000)
    r0 = 1.0 + (2.0 * st.uniform53(2000) - 1.0) * 2.5 * h
    s = np.sqrt(1.0 - z0 * z0)
    P0 = (np.stack([s * np.cos(az), s * np.sin(az), z0], 1) * r0[:, None]).astype(np.float32)
    (xk, yk, zk), _ = oracle.relax(spec, G.cell_pkg, G.nbr, fields, P0[:, 0], P0[:, 1], P0[:, 2], 50, 0.1)
    PK = np.stack([xk, yk, zk], 1).astype(np.float64)
    r = np.linalg.norm(PK, axis=1)
    # 15 clipped steps bring |d| under h, 35 more shrink it by 0.9^35; the
    # trilinear interpolation of |x| - 1 is off by about 3 h^2 / 8
    assert np.max(np.abs(r - 1.0)) < 0.1 * h
    u0 = P0.astype(np.float64) / np.linalg.norm(P0.astype(np.float64), axis=1)[:, None]
    assert np.max(np.linalg.norm(PK / r[:, None] - u0, axis=1)) < 1e-3


def test_relax_inputs_in_band():
    """The batch relaxation's particles lie within band_cells coarse cells
    (plus jitter) of their body's surface, and the split follows offsets."""
    bodies = si.random_bodies(6, seed=1)
    x, y, z, off = si.relax_particles(bodies, 60_000, seed=5)
    assert off[0] == 0 and off[-1] == 60_000 and np.all(np.diff(off) >= 0)
    for b, (shape, spec, _) in enumerate(bodies):
        sl = slice(off[b], off[b + 1])
        d = oracle.sdf(shape, x[sl], y[sl], z[sl])
        assert np.max(np.abs(d)) <= 2.0 * spec.lc + np.sqrt(3.0) * 0.5 * spec.h + 1e-6
        # both sides of the surface are covered (coarse bodies can be thinner
        # than the band inside)
        assert np.min(d) < -0.25 * spec.lc and np.max(d) > 1.5 * spec.lc
