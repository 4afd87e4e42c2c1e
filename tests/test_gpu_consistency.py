"""Consistency (sign) correction on the GPU against the oracle.

Noise as in the oracle pins: in random packages every value at |phi| >= 2h
changes sign (the point mask is taken from the oracle's values so that both
sides flip the same points), random far cells swap inside <-> outside.  The
device must restore its own clean grid bit for bit (phi, cell table,
neighbour and face tables), report the same counts as the oracle, and agree
with the oracle step-wise on the same float32 input.
"""
import numpy as np
import pytest

import oracle
import sg_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11473_b300 import build
    build.build()
    import paper_2512_11473_b300 as m
    return m


def H(t):
    return t.detach().cpu().numpy()


BODIES = {
    "sphere": lambda: si.sphere_small(),
    "torus": lambda: (si.torus(0.5, 0.2, rot=si.random_rotation(si.Stream(3))),
                      si.GridSpec((-0.9, -0.9, -0.9), (22, 22, 22), 0.02)),
    "rounded_box": lambda: (si.rounded_box((0.6, 0.45, 0.3), 0.06, rot=si.random_rotation(si.Stream(5))),
                            si.GridSpec((-1.0, -1.0, -1.0), (25, 25, 25), 0.02)),
    "torus_h0.002": lambda: si.torus_large(),
    # x-rows of exactly two 32-cell words: the cell flood's bit planes without padding bits
    "sphere_64x40x33": lambda: (si.sphere(0.5, centre=(0.05, -0.03, 0.02)),
                                si.GridSpec((-1.6, -1.0, -0.8), (64, 40, 33), 0.0125)),
    # x-rows of 10 words (300 cells, the last one 12 bits wide)
    "sphere_300x20x20": lambda: (si.sphere(0.1, centre=(0.31, 0.005, -0.004)),
                                 si.GridSpec((-3.0, -0.2, -0.2), (300, 20, 20), 0.005)),
}


def _setup(sg, name, seed=17, frac=0.3):
    shape, spec = BODIES[name]()
    g = sg.Grid(spec)
    P = g.tag_allocate(shape)
    g.init_sdf(shape)
    O = oracle.build_grid(spec, shape)
    assert P == O.P
    clean = {k: g.field(k).clone() for k in ("phi", "cell_pkg", "nbr")}
    pk, cells = si.sign_noise_masks(P, spec.n_cells, seed=seed, frac_pkg=frac, frac_cell=frac)
    flip = pk[:, None] & (np.abs(O.phi) >= 2.0 * spec.h)
    far = cells & (O.cell_pkg < 2)
    return shape, spec, g, O, clean, flip, far


def _apply_noise_device(g, flip, far):
    phi = g.field("phi")
    f = torch.from_numpy(flip).cuda()
    phi[f] = -phi[f]
    cp = g.field("cell_pkg")
    m = torch.from_numpy(far).cuda()
    cp[m] = 1 - cp[m]
    torch.cuda.synchronize()


@pytest.mark.parametrize("name", ["sphere", "torus", "rounded_box", "sphere_64x40x33", "sphere_300x20x20",
                                  "torus_h0.002"])
def test_consistency_restores_and_matches_oracle(sg, name):
    shape, spec, g, O, clean, flip, far = _setup(sg, name, frac=0.3 if name != "torus_h0.002" else 0.2)
    faces0 = H(g.field("nbr"))[:, [12, 14, 10, 16, 4, 22]]
    _apply_noise_device(g, flip, far)
    noisy_phi = H(g.field("phi")).astype(np.float64)
    noisy_cp = H(g.field("cell_pkg"))
    out = g.consistency_correct(1.0)
    assert out[0] == int(flip.sum()) and out[1] == int(far.sum())
    assert torch.equal(g.field("phi"), clean["phi"])
    assert torch.equal(g.field("cell_pkg"), clean["cell_pkg"])
    assert torch.equal(g.field("nbr"), clean["nbr"])
    assert np.array_equal(H(g.field("nbr"))[:, [12, 14, 10, 16, 4, 22]], faces0)
    g.check_tables()  # the rebuilt neighbour and face tables agree with the cells
    g.sync()
    # step-wise: the oracle on the device's noisy float32 input
    cp2, nb2, phi2, ch, sw = oracle.consistency_correct(spec, O.P, noisy_cp, O.pkg_cell, O.pkg_type, O.nbr,
                                                        noisy_phi, sweeps=True)
    assert ch == (out[0], out[1])
    assert sw == (out[2], out[3])  # the same floods, sweep for sweep
    assert np.array_equal(phi2.astype(np.float32), H(g.field("phi")))
    assert np.array_equal(cp2, H(g.field("cell_pkg")))
    assert np.array_equal(nb2, H(g.field("nbr")))
    # the face stencils read the rebuilt face table: a gradient equals the clean grid's
    g.gradient()
    gx = g.field("gx").clone()
    g2 = sg.Grid(spec)
    g2.tag_allocate(shape)
    g2.init_sdf(shape)
    g2.gradient()
    assert torch.equal(gx, g2.field("gx"))


def test_consistency_clean_grid_unchanged(sg):
    shape, spec, g, O, clean, _, _ = _setup(sg, "torus")
    out = g.consistency_correct(1.0)
    assert out[:2] == (0, 0)
    for k, v in clean.items():
        assert torch.equal(g.field(k), v)


def test_consistency_bad_trust(sg):
    shape, spec, g, O, clean, _, _ = _setup(sg, "sphere")
    for t in (0.0, -1.0, float("nan")):
        with pytest.raises(sg.SgError):
            g.consistency_correct(t)


def test_flood_barrier_wait_gives_up(sg):
    """A CTA that never reaches the persistent floods' grid barrier: the
    bounded waits give up, the call reports SG_ERR_TIMEOUT, nothing changed,
    and the grid (and the context) still work.  The give-up time is measured
    (2^21 polls of at least 32 ns each: no less than 67 ms)."""
    import time
    shape, spec = BODIES["sphere"]()
    g = sg.Grid(spec)
    g.tag_allocate(shape)
    g.init_sdf(shape)
    before = {k: g.field(k).clone() for k in ("phi", "cell_pkg", "nbr")}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with pytest.raises(sg.SgError) as e:
        g.debug_consistency_absent_cta(1.0)
    dt = time.perf_counter() - t0
    print("barrier wait gave up after %.3f s" % dt)
    assert 0.05 < dt < 10.0
    assert e.value.status == sg.SG_ERR_TIMEOUT
    for k, v in before.items():
        assert torch.equal(g.field(k), v), k
    out = g.consistency_correct(1.0)
    assert out[:2] == (0, 0)
    for k, v in before.items():
        assert torch.equal(g.field(k), v), k
    g.close()


def test_cell_flood_give_up_leaves_grid_unchanged(sg):
    """The point flood settles, the cell flood's barrier cannot complete: the
    call reports SG_ERR_TIMEOUT and neither phi nor the tables changed (the
    signs are applied only after both floods settled)."""
    shape, spec, g, O, clean, flip, far = _setup(sg, "sphere")
    _apply_noise_device(g, flip, far)
    noisy = {k: g.field(k).clone() for k in ("phi", "cell_pkg", "nbr")}
    with pytest.raises(sg.SgError) as e:
        g.debug_consistency(1.0, sg.DEBUG_CC_ABSENT_CELLS)
    assert e.value.status == sg.SG_ERR_TIMEOUT
    for k, v in noisy.items():
        assert torch.equal(g.field(k), v), k
    out = g.consistency_correct(1.0)  # and the grid still corrects
    assert out[0] == int(flip.sum()) and out[1] == int(far.sum())
    for k, v in clean.items():
        assert torch.equal(g.field(k), v), k


@pytest.mark.parametrize("name", ["sphere", "sphere_64x40x33", "torus"])
def test_per_sweep_floods_match_persistent_and_oracle(sg, name):
    """The floods of devices without cooperative launch (a launch per sweep,
    flags read by the host in batches): the same corrected grid, counts and
    sweep counts as the persistent floods and as the oracle."""
    shape, spec, g, O, clean, flip, far = _setup(sg, name)
    _apply_noise_device(g, flip, far)
    noisy_phi = H(g.field("phi")).astype(np.float64)
    noisy_cp = H(g.field("cell_pkg"))
    out = g.debug_consistency(1.0, sg.DEBUG_CC_PER_SWEEP)
    for k, v in clean.items():
        assert torch.equal(g.field(k), v), k
    cp2, nb2, phi2, ch, sw = oracle.consistency_correct(spec, O.P, noisy_cp, O.pkg_cell, O.pkg_type, O.nbr,
                                                        noisy_phi, sweeps=True)
    assert ch == (out[0], out[1])
    assert sw == (out[2], out[3])
    # the persistent path on the same noise
    _apply_noise_device(g, flip, far)
    assert g.consistency_correct(1.0) == out


def test_debug_consistency_flags(sg):
    shape, spec, g, O, clean, _, _ = _setup(sg, "sphere")
    for bad in (8, -1, sg.DEBUG_CC_ABSENT_POINTS | sg.DEBUG_CC_PER_SWEEP):
        with pytest.raises(sg.SgError) as e:
            g.debug_consistency(1.0, bad)
        assert e.value.status == sg.SG_ERR_INVALID
