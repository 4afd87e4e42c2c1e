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
