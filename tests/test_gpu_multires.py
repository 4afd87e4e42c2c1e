"""Multi-resolution tagging on the GPU.

Every layer of a stack built coarse to fine (sg_tag_allocate_from) must
equal the same layer tagged in full (sg_tag_allocate) and the oracle's
layer, bit for bit, with the oracle's count of distance evaluations; the
level sets of every layer match the oracle within 1e-4 h.
"""
import numpy as np
import pytest

import oracle
import sg_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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
TABLES = ("cell_pkg", "pkg_cell", "pkg_type", "nbr")


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


def _check_stack(sg, shape, spec, layers, with_oracle=True):
    M = sg.MultiResolution(spec, shape, layers=layers)
    O = oracle.build_layers(spec, shape, layers) if with_oracle else None
    for k, g in enumerate(M.grids):
        full = sg.Grid(g.spec)
        assert full.tag_allocate(shape) == g.P
        for t in TABLES:
            assert torch.equal(g.field(t), full.field(t)), (k, t)
        full.close()
        if O is not None:
            assert g.P == O[k].P
            assert np.array_equal(H(g.field("cell_pkg")), O[k].cell_pkg)
            assert np.array_equal(H(g.field("nbr")), O[k].nbr)
            assert M.evaluated[k] == O[k].evaluated
            assert np.max(np.abs(H(g.field("phi")).astype(np.float64) - O[k].phi)) <= 1e-4 * g.spec.h
    return M


@pytest.mark.parametrize("name", sorted(CASES))
def test_layers_equal_full_and_oracle(sg, name):
    shape, spec = CASES[name]
    _check_stack(sg, shape, spec, 3).close()


def test_shelled_sphere_full_stack(sg):
    """The paper's Table 1 body at h = 1/1024: six layers from 8^3 coarse
    cells; every layer equals full tagging, the finest also the oracle's."""
    shape, spec = si.shelled_sphere()
    L = sg.multires_layers(spec)
    assert L == 6
    M = _check_stack(sg, shape, spec, L, with_oracle=False)
    O = oracle.build_grid(spec, shape)
    g = M.finest
    assert g.P == O.P
    assert np.array_equal(H(g.field("cell_pkg")), O.cell_pkg)
    assert np.array_equal(H(g.field("nbr")), O.nbr)
    assert M.evaluated[-1] < spec.n_cells // 8
    M.close()


def test_mismatched_coarse_layer_refused(sg):
    shape, spec = CASES["sphere"]
    coarse = sg.Grid(oracle.coarser(spec))
    fine = sg.Grid(spec)
    with pytest.raises(sg.SgError):  # coarse layer not initialised
        fine.tag_allocate_from(coarse, shape)
    coarse.tag_allocate(shape)
    coarse.init_sdf(shape)
    other = sg.Grid(si.GridSpec(spec.lo, (30, 32, 32), spec.h))
    with pytest.raises(sg.SgError):  # dims are not twice the coarse dims
        other.tag_allocate_from(coarse, shape)
    shifted = sg.Grid(si.GridSpec((-0.99, -1.0, -1.0), spec.dims, spec.h))
    with pytest.raises(sg.SgError):  # another origin
        shifted.tag_allocate_from(coarse, shape)
    P, ev = fine.tag_allocate_from(coarse, shape)
    assert P > 2 and 0 < ev < spec.n_cells
