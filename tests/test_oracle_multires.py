"""Pins of the oracle's multi-resolution tagging.

A layer tagged from its coarser layer (distances evaluated only in fine
cells covered by coarse core cells, the far side of every other cell taken
from the coarse layer) must equal the layer tagged in full, bit for bit:
a fine cell inside a coarse cell that is not core lies at least 0.57 coarse
cells = 1.13 fine cells from the surface, so it cannot be core, and its
side is the coarse cell's side.
"""
import numpy as np
import pytest

import oracle
import sg_inputs as si

CASES = {
    "sphere": (si.sphere(0.7, centre=(0.03, -0.02, 0.01)), si.GridSpec((-1.0, -1.0, -1.0), (32, 32, 32), 1.0 / 64)),
    "torus": (si.torus(0.5, 0.18, rot=si.random_rotation(si.Stream(3))),
              si.GridSpec((-0.8, -0.8, -0.8), (32, 32, 32), 0.0125)),
    "rounded_box": (si.rounded_box((0.6, 0.45, 0.3), 0.06, rot=si.random_rotation(si.Stream(5))),
                    si.GridSpec((-1.0, -1.0, -1.0), (40, 40, 40), 0.0125)),
    "prism": (si.prism(((0.0, 0.0), (1.0, 0.0), (0.3, 0.8)), 0.0, 1.0),
              si.GridSpec((-0.2, -0.2, -0.2), (28, 24, 28), 0.0125)),
    "shell": (si.shell(0.3, 0.31, (0.5, 0.5, 0.5)), si.GridSpec((0.0, 0.0, 0.0), (64, 64, 64), 1.0 / 256)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_layers_equal_full_tagging(name):
    shape, spec = CASES[name]
    layers = oracle.build_layers(spec, shape, 3)
    assert [L.spec.dims for L in layers][-1] == tuple(spec.dims)
    for k, L in enumerate(layers):
        full = oracle.build_grid(L.spec, shape)
        assert L.P == full.P, k
        assert np.array_equal(L.cell_pkg, full.cell_pkg), k
        assert np.array_equal(L.cell_type, full.cell_type), k
        assert np.array_equal(L.nbr, full.nbr), k
        assert np.array_equal(L.phi, full.phi), k
        if k:
            coarse = layers[k - 1]
            # evaluations: the 8 fine cells of every coarse core cell
            assert L.evaluated == 8 * int(np.sum(coarse.cell_type == 2))


def test_layer_spec_halving():
    spec = si.GridSpec((0.0, 0.0, 0.0), (64, 32, 16), 1.0 / 256)
    c = oracle.coarser(spec)
    assert c.dims == (32, 16, 8) and c.h == 2.0 / 256 and c.lo == spec.lo
    assert np.allclose(c.hi(), spec.hi())
