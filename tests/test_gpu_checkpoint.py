"""Checkpoint and restore of a grid and of the surrogate network.

The tables and fields of a grid go to a file and back into a fresh grid of
the same description bit for bit; the restored grid then computes what the
original computes (a reinit sweep, the integrals and a probe, bit for bit);
corrupted tables are refused.  The network's FP32 master vector round-trips
and its BF16 copy is the rounding the tensor cores use.
"""
import numpy as np
import pytest

import sg_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAMES = ("phi", "gx", "gy", "gz", "W", "Gx", "Gy", "Gz")


@pytest.fixture(scope="module")
def sg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11473_b300 import build
    build.build()
    import paper_2512_11473_b300 as m
    return m


def _grid(sg):
    shape = si.torus(0.45, 0.15, rot=si.random_rotation(si.Stream(21)))
    spec = si.GridSpec((-0.8,) * 3, (20, 20, 20), 0.02)
    g = sg.Grid(spec)
    g.tag_allocate(shape)
    g.init_sdf(shape)
    g.reinit(10, 0.5)
    g.gradient()
    g.kernel_integrals()
    return spec, g


def test_grid_checkpoint_round_trip(sg, tmp_path):
    spec, g = _grid(sg)
    path = tmp_path / "ck.npz"
    sg.save_checkpoint(path, grid=g)
    h = sg.Grid(spec)
    sg.load_checkpoint(path, grid=h)
    assert h.P == g.P
    for name in ("cell_pkg", "pkg_cell", "pkg_type", "nbr") + NAMES:
        assert torch.equal(h.field(name), g.field(name)), name
    h.check_tables()
    h.sync()
    # the restored grid computes what the original computes
    x, y, z = si.box_particles(20_000, spec.lo, spec.hi(), seed=5)
    X = [torch.from_numpy(v).cuda() for v in (x, y, z)]
    for grid in (g, h):
        grid.reinit(1, 0.5)
        grid.kernel_integrals()
    for name in ("phi", "W", "Gx"):
        assert torch.equal(h.field(name), g.field(name)), name
    a, b = g.probe(*X, morton=True), h.probe(*X, morton=True)
    for k in a:
        assert torch.equal(a[k], b[k]), k


def test_restore_refuses_inconsistent_tables(sg):
    spec, g = _grid(sg)
    ck = g.checkpoint()
    bad = dict(ck)
    bad["nbr"] = ck["nbr"].copy()
    bad["nbr"][5, 3] = int(ck["P"]) + 7  # a neighbour id beyond the packages
    h = sg.Grid(spec)
    with pytest.raises(sg.SgError) as e:
        h.restore(bad)
    assert e.value.status == sg.SG_ERR_INVALID
    bad = dict(ck)
    bad["pkg_cell"] = ck["pkg_cell"].copy()
    bad["pkg_cell"][[3, 4]] = bad["pkg_cell"][[4, 3]]  # the cell table no longer points back
    with pytest.raises(sg.SgError) as e:
        h.restore(bad)
    assert e.value.status == sg.SG_ERR_INVALID
    h.restore(ck)  # and the grid takes a good checkpoint afterwards
    assert torch.equal(h.field("phi"), g.field("phi"))


def test_mlp_checkpoint_round_trip(sg, tmp_path):
    par = si.mlp_init_params(21)
    net = sg.MLP(par)
    x = torch.randn(1000, 32).clamp(-1, 1).to(torch.bfloat16).cuda()
    x[:, 27:] = 0
    path = tmp_path / "net.npz"
    sg.save_checkpoint(path, mlp=net)
    d = np.load(path)
    assert np.array_equal(d["mlp_master"], net.get_params())
    bf = torch.from_numpy(d["mlp_master"]).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(d["mlp_bf16"], bf)
    other = sg.MLP(si.mlp_init_params(22))
    sg.load_checkpoint(path, mlp=other)
    assert torch.equal(other.forward(x), net.forward(x))
