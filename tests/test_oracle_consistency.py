"""Pins of the oracle's consistency (sign) correction.

The input is a clean grid (analytic signed distances) corrupted by synthetic
sign noise: in random packages every value at |phi| >= 2h changes sign, and
random far cells swap their far package (inside <-> outside).  Signs within
h of the surface are trusted and untouched, and the magnitudes are right, so
the 1-Lipschitz bound of a distance makes the correction exact: every sign
and every far cell must come back to the clean grid, bit for bit, with the
neighbour table rebuilt to match; a clean grid is left unchanged.
"""
import numpy as np
import pytest

import oracle
import sg_inputs as si


def _noisy(G, seed, frac=0.3):
    h = G.spec.h
    pk, cells = si.sign_noise_masks(G.P, G.spec.n_cells, seed=seed, frac_pkg=frac, frac_cell=frac)
    phi = G.phi.copy()
    flip = pk[:, None] & (np.abs(phi) >= 2.0 * h)
    phi[flip] = -phi[flip]
    cp = G.cell_pkg.copy()
    far = cells & (cp < 2)
    cp[far] = 1 - cp[far]
    return phi, cp, int(flip.sum()), int(far.sum())


BODIES = {
    "sphere": lambda: si.sphere_small(),
    "torus": lambda: (si.torus(0.5, 0.2, rot=si.random_rotation(si.Stream(3))),
                      si.GridSpec((-0.9, -0.9, -0.9), (22, 22, 22), 0.02)),
    "rounded_box": lambda: (si.rounded_box((0.6, 0.45, 0.3), 0.06, rot=si.random_rotation(si.Stream(5))),
                            si.GridSpec((-1.0, -1.0, -1.0), (25, 25, 25), 0.02)),
}


@pytest.mark.parametrize("name", sorted(BODIES))
def test_consistency_restores_clean_grid(name):
    shape, spec = BODIES[name]()
    G = oracle.build_grid(spec, shape)
    phi, cp, n_flip, n_far = _noisy(G, seed=17)
    assert n_flip > 100 and n_far > 10
    cp2, nb2, phi2, ch = oracle.consistency_correct(spec, G.P, cp, G.pkg_cell, G.pkg_type, G.nbr, phi)
    assert np.array_equal(cp2, G.cell_pkg)
    assert np.array_equal(nb2, G.nbr)
    assert np.array_equal(phi2, G.phi)
    assert ch == (n_flip, n_far)


@pytest.mark.parametrize("name", sorted(BODIES))
def test_consistency_clean_grid_unchanged(name):
    shape, spec = BODIES[name]()
    G = oracle.build_grid(spec, shape)
    cp2, nb2, phi2, ch = oracle.consistency_correct(spec, G.P, G.cell_pkg, G.pkg_cell, G.pkg_type, G.nbr, G.phi)
    assert ch == (0, 0)
    assert np.array_equal(phi2, G.phi) and np.array_equal(cp2, G.cell_pkg) and np.array_equal(nb2, G.nbr)


def test_consistency_signs_match_distance():
    """After the correction every active value has the sign of the closed-form
    distance at its data point (torus, also inside its hole)."""
    shape, spec = BODIES["torus"]()
    G = oracle.build_grid(spec, shape)
    phi, cp, _, _ = _noisy(G, seed=23, frac=0.5)
    _, _, phi2, _ = oracle.consistency_correct(spec, G.P, cp, G.pkg_cell, G.pkg_type, G.nbr, phi)
    nx, ny, _ = spec.dims
    pc = G.pkg_cell[2:].astype(np.int64)
    I, J, K = pc % nx, (pc // nx) % ny, pc // (nx * ny)
    d = np.arange(64)
    pts = [spec.lo[a] + (4 * c[:, None] + v[None, :] + 0.5) * spec.h
           for a, (c, v) in enumerate(((I, d % 4), (J, (d // 4) % 4), (K, d // 16)))]
    ref = oracle.sdf(shape, pts[0].ravel(), pts[1].ravel(), pts[2].ravel())
    got = phi2[2:].ravel()
    nz = ref != 0
    assert np.array_equal(np.sign(got[nz]), np.sign(ref[nz]))


def test_consistency_trusted_band_is_kept():
    """Values with |phi| < h are taken as given: a wrong sign planted there
    stays (the correction trusts that band by definition)."""
    shape, spec = si.sphere_small()
    G = oracle.build_grid(spec, shape)
    phi = G.phi.copy()
    near = np.argwhere((np.abs(phi) < 0.5 * spec.h) & (np.arange(G.P)[:, None] >= 2))
    p, e = near[0]
    phi[p, e] = -phi[p, e]
    _, _, phi2, ch = oracle.consistency_correct(spec, G.P, G.cell_pkg, G.pkg_cell, G.pkg_type, G.nbr, phi)
    assert phi2[p, e] == phi[p, e]


def _flood_depth(n, edges_a, edges_b, seeds, passable):
    """1 + the largest graph distance from the seeds over passable entries
    (multi-source breadth-first search on the face-neighbour graph): the
    number of Jacobi sweeps of a flood whose fronts never meet, the last one
    labelling nothing."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import dijkstra
    keep = passable[edges_a] & passable[edges_b]
    A = coo_matrix((np.ones(int(keep.sum())), (edges_a[keep], edges_b[keep])), shape=(n, n)).tocsr()
    d = dijkstra(A, directed=False, indices=np.flatnonzero(seeds), unweighted=True, min_only=True)
    d = d[passable & np.isfinite(d)]
    return 1 + int(d.max())


@pytest.mark.parametrize("name", sorted(BODIES))
def test_consistency_sweep_counts_are_flood_depths(name):
    """On a clean grid the two floods' sweep counts equal one plus the
    largest breadth-first distance from their seeds: the points from the
    trusted band through the active packages, the cells from the inner
    cells through the far cells (core cells block)."""
    shape, spec = BODIES[name]()
    G = oracle.build_grid(spec, shape)
    *_, ch, sw = oracle.consistency_correct(spec, G.P, G.cell_pkg, G.pkg_cell, G.pkg_type, G.nbr, G.phi, sweeps=True)
    assert ch == (0, 0)
    # points: graph over the active packages' data points, face neighbours from the 27-entry table
    P, h = G.P, spec.h
    tau = float(np.float32(float(np.float32(1.0)) * h))
    d = np.arange(64)
    i, j, k = d % 4, (d // 4) % 4, d // 16
    ea, eb = [], []
    for axis in range(3):
        loc = (i, j, k)[axis]
        up = loc == 3  # the +axis neighbour lies in the next package
        step = (1, 4, 16)[axis]
        slot = 13 + (1, 3, 9)[axis]
        for p in range(2, P):
            inner = ~up
            ea.append(p * 64 + d[inner])
            eb.append(p * 64 + d[inner] + step)
            q = G.nbr[p, slot]
            if q >= 2:
                ea.append(p * 64 + d[up])
                eb.append(q * 64 + d[up] - 3 * step)
    ea, eb = np.concatenate(ea), np.concatenate(eb)
    n = P * 64
    phi = G.phi.reshape(-1)
    active = np.zeros(n, bool)
    active[128:] = True
    seeds = active & (np.abs(phi) < tau) & (phi != 0)
    assert sw[0] == _flood_depth(n, ea, eb, seeds, active)
    # cells: graph over the background mesh, core cells removed
    nx, ny, nz = spec.dims
    c = np.arange(nx * ny * nz).reshape(nz, ny, nx)
    pairs = [(c[:, :, :-1], c[:, :, 1:]), (c[:, :-1, :], c[:, 1:, :]), (c[:-1, :, :], c[1:, :, :])]
    ca = np.concatenate([a.ravel() for a, _ in pairs])
    cb = np.concatenate([b.ravel() for _, b in pairs])
    cp = G.cell_pkg
    core = (cp >= 2) & (G.pkg_type[np.maximum(cp, 0)] == 2)
    seeds_c = (cp >= 2) & ~core
    assert sw[1] == _flood_depth(cp.size, ca, cb, seeds_c, ~core)
