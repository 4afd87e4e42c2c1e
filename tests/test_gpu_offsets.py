"""The 64-bit address kernels against the 32-bit offset kernels.

The probe, the exact kernel integrals and the relaxation steps run on
32-bit byte offsets while the store allows (fewer than 2^24 packages and
2^30 particles for the probe and the integrals, 2^21 packages for the
relaxation's table) and on 64-bit addresses beyond.  Stores that large do
not fit a test, so the testing hook sg_debug_wide_offsets forces the 64-bit
kernels on ordinary inputs: both must give the same bits, and the 32-bit
kernels are themselves held to the oracle by the parity tests.
"""
import pytest

import sg_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OUTS = ("phi", "nx", "ny", "nz", "W", "Gx", "Gy", "Gz")


@pytest.fixture(scope="module")
def sg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11473_b300 import build
    build.build()
    import paper_2512_11473_b300 as m
    yield m
    m.debug_wide_offsets(False)


def _grid(sg, shape, spec):
    g = sg.Grid(spec)
    g.tag_allocate(shape)
    g.init_sdf(shape)
    g.reinit(10, 0.5)
    g.gradient()
    return g


@pytest.mark.parametrize("morton", [True, False])
def test_probe_and_integrals_wide_equal(sg, morton):
    shape = si.torus(0.45, 0.15, rot=si.random_rotation(si.Stream(31)))
    spec = si.GridSpec((-0.8,) * 3, (40, 40, 40), 0.01)
    g = _grid(sg, shape, spec)
    x, y, z = si.box_particles(300_000, spec.lo, spec.hi(), seed=9)  # inside, near and outside the band
    X = [torch.from_numpy(v).cuda() for v in (x, y, z)]
    res = []
    for wide in (False, True):
        sg.debug_wide_offsets(wide)
        g.kernel_integrals()
        fields = {f: g.field(f).clone() for f in ("W", "Gx", "Gy", "Gz")}
        res.append((fields, g.probe(*X, morton=morton)))
    sg.debug_wide_offsets(False)
    (f0, p0), (f1, p1) = res
    for k in f0:
        assert torch.equal(f0[k], f1[k]), k
    for k in p0:
        assert torch.equal(p0[k], p1[k]), k
    g.close()


def test_relax_wide_equal(sg):
    bodies = si.random_bodies(4, seed=3, p_lo=1e2, p_hi=2e3)
    x, y, z, off = si.relax_particles(bodies, 60_000, seed=7)
    X0 = [torch.from_numpy(v).cuda() for v in (x, y, z)]
    res = []
    for wide in (False, True):
        sg.debug_wide_offsets(wide)  # read when the relaxation graph is recorded: a fresh batch each time
        grids = []
        for shape, spec, _ in bodies:
            g = sg.Grid(spec)
            g.tag_allocate(shape)
            g.init_sdf(shape)
            grids.append(g)
        batch = sg.Batch(grids)
        for g in grids:
            g.close()
        Y = [v.clone() for v in X0]
        out = {k: torch.full_like(Y[0], float("nan")) for k in OUTS}
        batch.relax(*Y, off, 5, 0.1, plan=sg.make_plan(4, 1, 10, 0.5), sweeps=True, out=out)
        torch.cuda.synchronize()
        res.append((Y, out))
        batch.close()
    sg.debug_wide_offsets(False)
    (y0, o0), (y1, o1) = res
    for a, b in zip(y0, y1):
        assert torch.equal(a, b)
    for k in OUTS:
        assert torch.equal(o0[k], o1[k]), k
