"""The paper's own benchmark workload ("Performance Evaluation", Table 1):
the shelled sphere (centre (0.5, 0.5, 0.5), radii 0.3 and 0.31) at resolution
1/1024, a sequential update of every active value and the 7-point Laplacian.
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


@pytest.mark.parametrize("h", [1.0 / 256, 1.0 / 1024])
def test_shell_tags_phi_sequential_laplacian(sg, h):
    shape, spec = si.shelled_sphere(h)
    g = sg.Grid(spec)
    P = g.tag_allocate(shape)
    g.init_sdf(shape)
    O = oracle.build_grid(spec, shape)
    assert O.near_ties == 0 and P == O.P
    assert np.array_equal(H(g.field("cell_pkg")), O.cell_pkg)
    assert np.array_equal(H(g.field("nbr")), O.nbr)
    phi32 = H(g.field("phi"))
    assert np.max(np.abs(phi32.astype(np.float64) - O.phi)) <= 1e-4 * spec.h
    g.sequential_update(1e-6)
    assert np.array_equal(H(g.field("phi")), oracle.sequential(phi32, 1e-6))
    g.laplacian()
    phi = H(g.field("phi")).astype(np.float64)
    ref = oracle.laplacian(spec, O.nbr, phi)
    tol = 8 * float(np.finfo(np.float32).eps) * oracle.far_value(spec) / spec.h ** 2
    assert np.max(np.abs(H(g.field("lap")) - ref)) <= tol
    g.sync()
