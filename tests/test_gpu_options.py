"""The grid options on the GPU against the oracle: kernel support and
Heaviside half width of the integrals, Morton package ids, and the errors
for options a call cannot take."""
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


def _with(spec, **kw):
    d = dict(kernel_support=spec.kernel_support, heaviside_eps=spec.heaviside_eps, id_order=spec.id_order)
    d.update(kw)
    return si.GridSpec(spec.lo, spec.dims, spec.h, **d)


BODIES = {
    "sphere": si.sphere_small,
    "torus": lambda: (si.torus(0.5, 0.18, rot=si.random_rotation(si.Stream(3))),
                      si.GridSpec((-0.8, -0.8, -0.8), (16, 16, 16), 0.025)),
}


@pytest.mark.parametrize("name", sorted(BODIES))
@pytest.mark.parametrize("R,e", [(1.5, 1.0), (2.0, 0.5), (2.5, 1.0), (3.0, 2.0)])
def test_integrals_support_and_eps(sg, name, R, e):
    shape, spec0 = BODIES[name]()
    spec = _with(spec0, kernel_support=R * spec0.h, heaviside_eps=e * spec0.h)
    g = sg.Grid(spec)
    g.tag_allocate(shape)
    g.init_sdf(shape)
    g.reinit(10, 0.5)
    g.kernel_integrals()
    O = oracle.build_grid(spec, shape)
    phi = H(g.field("phi")).astype(np.float64)
    ref = oracle.kernel_integrals(spec, O.nbr, phi)
    for a, f in enumerate(("W", "Gx", "Gy", "Gz")):
        assert np.max(np.abs(H(g.field(f)) - ref[a])) <= 1e-5, (f, R, e)


@pytest.mark.parametrize("name", sorted(BODIES))
def test_morton_ids(sg, name):
    shape, spec0 = BODIES[name]()
    spec1 = _with(spec0, id_order=1)
    A, B = sg.Grid(spec0), sg.Grid(spec1)
    for g, sp in ((A, spec0), (B, spec1)):
        g.tag_allocate(shape)
        O = oracle.build_grid(sp, shape)
        for t in ("cell_pkg", "pkg_cell", "pkg_type", "nbr"):
            assert np.array_equal(H(g.field(t)), getattr(O, t)), (sp.id_order, t)
    # a relabelling: the per-cell results of the whole chain are the same bits
    for g in (A, B):
        g.init_sdf(shape)
        g.gradient()
        g.reinit(12, 0.5)
        g.kernel_integrals()
    ca, cb = H(A.field("cell_pkg")), H(B.field("cell_pkg"))
    act = ca >= 2
    perm = np.empty(A.P, np.int64)
    perm[:2] = [0, 1]
    perm[ca[act]] = cb[act]
    for f in ("phi", "gx", "gy", "gz", "W", "Gx", "Gy", "Gz"):
        assert np.array_equal(H(A.field(f)), H(B.field(f))[perm]), f
    x, y, z = si.sphere_shell_particles(20000, 0.7, 0.1, seed=3)
    X = [torch.from_numpy(v).cuda() for v in (x, y, z)]
    pa, pb = A.probe(*X, morton=True), B.probe(*X, morton=True)
    for k in pa:
        assert torch.equal(pa[k], pb[k]), k


def test_morton_ids_in_layers(sg):
    shape, spec = si.shell(0.3, 0.31, (0.5, 0.5, 0.5)), si.GridSpec((0.0, 0.0, 0.0), (64, 64, 64), 1.0 / 256, id_order=1)
    M = sg.MultiResolution(spec, shape, layers=3)
    for g in M.grids:
        full = sg.Grid(g.spec)
        full.tag_allocate(shape)
        for t in ("cell_pkg", "pkg_cell", "nbr"):
            assert torch.equal(g.field(t), full.field(t)), t
        full.close()
    M.close()


def test_option_errors(sg):
    shape, spec = si.sphere_small()
    for bad in (dict(kernel_support=3.5 * spec.h), dict(kernel_support=-1.0), dict(heaviside_eps=-0.1),
                dict(id_order=2)):
        with pytest.raises(sg.SgError):
            sg.Grid(_with(spec, **bad))
    g = sg.Grid(_with(spec, kernel_support=3.0 * spec.h))
    g.tag_allocate(shape)
    g.init_sdf(shape)
    net = sg.MLP(si.mlp_init_params(4))
    with pytest.raises(sg.SgError):  # the surrogate is defined for support 2h and eps = h
        g.kernel_integrals(mode=1, mlp=net)
    # batches share one tap table: one support (at most 2h) for all bodies
    g2 = sg.Grid(_with(spec, kernel_support=1.5 * spec.h))
    g2.tag_allocate(shape)
    g2.init_sdf(shape)
    g3 = sg.Grid(spec)
    g3.tag_allocate(shape)
    g3.init_sdf(shape)
    with pytest.raises(sg.SgError):
        sg.Batch([g2, g3])
    with pytest.raises(sg.SgError):
        sg.Batch([g])
    net.close()


def test_batch_with_eps_equals_single(sg):
    bodies = [(s, _with(sp, heaviside_eps=0.5 * sp.h)) for s, sp, _ in si.random_bodies(4, seed=1, p_lo=1e2, p_hi=2e3)]
    grids, ref = [], []
    for shape, spec in bodies:
        g = sg.Grid(spec)
        g.tag_allocate(shape)
        g.init_sdf(shape)
        grids.append(g)
        r = sg.Grid(spec)
        r.tag_allocate(shape)
        r.init_sdf(shape)
        r.gradient()
        r.reinit(20, 0.5)
        r.kernel_integrals()
        ref.append(r.field("W").clone())
    b = sg.Batch(grids)
    b.run(sg.make_plan(4, 2, 20, 0.5))
    for i, w in enumerate(ref):
        assert torch.equal(b.field(i, "W"), w)
    b.close()


def test_check_tables_and_sticky_error(sg):
    """Tables edited through borrowed pointers: the device check finds an
    out-of-range neighbour id, a neighbour entry that names the wrong package
    and a cell whose package does not name it back; the word stays set until
    cleared.  No sweep runs on an edited table."""
    shape, spec = si.sphere_small()
    g = sg.Grid(spec)
    P = g.tag_allocate(shape)
    g.check_tables()
    g.sync()
    nbr, cp = g.field("nbr"), g.field("cell_pkg")
    act = torch.nonzero(cp >= 2).flatten()
    for edit in ("range", "neighbour", "cell"):
        nb0, cp0 = nbr.clone(), cp.clone()
        if edit == "range":
            nbr[5, 3] = P + 7
        elif edit == "neighbour":
            nbr[5, 3] = 5 if int(nbr[5, 3]) != 5 else 6
        else:
            c = int(act[10])
            cp[c] = int(cp[int(act[11])])
        g.check_tables()
        with pytest.raises(sg.SgError):
            g.sync()
        with pytest.raises(sg.SgError):  # sticky
            g.sync()
        nbr.copy_(nb0)
        cp.copy_(cp0)
        g.clear_error()
        g.check_tables()
        g.sync()
    g.close()


class _Budget:
    """A device-memory hook that refuses any allocation past a byte budget."""

    def __init__(self, sg, budget):
        self.budget, self.used, self.sizes = budget, 0, {}

        def _alloc(nbytes, stream, ctx):
            if self.used + nbytes > self.budget:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), device=0, stream=stream or 0)
            self.used += nbytes
            self.sizes[p] = nbytes
            return p

        def _free(ptr, nbytes, stream, ctx):
            self.used -= self.sizes.pop(ptr, 0)
            torch.cuda.caching_allocator_delete(ptr)

        self.alloc_fn, self.free_fn = sg.ALLOC_FN(_alloc), sg.FREE_FN(_free)
        self.struct = sg.sg_allocator(self.alloc_fn, self.free_fn, None)


def test_allocator_failure_is_reported(sg):
    """An allocator that runs dry gives SG_ERR_OOM, the grid keeps its previous
    state, later calls succeed once memory is there, and every byte is
    returned at the end."""
    shape, spec = si.sphere_small()
    B = _Budget(sg, 4096)
    g = sg.Grid(spec, allocator=B)
    with pytest.raises(sg.SgError) as e:
        g.tag_allocate(shape)  # cell tables do not fit
    assert e.value.status == 2
    with pytest.raises(sg.SgError) as e:
        g.init_sdf(shape)  # still untagged
    assert e.value.status == 4
    B.budget = 1 << 30
    P = g.tag_allocate(shape)
    assert P == 1634
    B.budget = B.used + 1000  # the level set (P x 64 floats) does not fit
    with pytest.raises(sg.SgError) as e:
        g.init_sdf(shape)
    assert e.value.status == 2
    B.budget = 1 << 30
    g.init_sdf(shape)
    g.gradient()
    ref = sg.Grid(spec)
    ref.tag_allocate(shape)
    ref.init_sdf(shape)
    ref.gradient()
    assert torch.equal(g.field("gx"), ref.field("gx"))
    ref.close()
    g.close()
    torch.cuda.synchronize()
    assert B.used == 0 and not B.sizes
