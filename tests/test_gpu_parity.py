"""GPU parity: every libsg step against the FP64 oracle on the same inputs.

Bars: tagging, ids, tables, Morton keys and order bit-exact; phi within
1e-4 h; gradients, kernel integrals, probe values within 1e-5 absolute (probe
normals where |grad| > 0.5).  "Step-wise" checks hand the GPU's float32
input, widened to double, to the oracle for one step; "end-to-end" checks run
both chains from their own start.
"""
import numpy as np
import pytest

import oracle
import sg_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS32 = float(np.finfo(np.float32).eps)


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


def _cases():
    rot1 = si.random_rotation(si.Stream(21))
    rot2 = si.random_rotation(si.Stream(22))
    return {
        "sphere_small": si.sphere_small(),
        "sphere_offset": (si.sphere(0.55, centre=(0.03, -0.02, 0.05)), si.GridSpec((-1.0,) * 3, (8, 8, 8), 0.0625)),
        "torus_rot": (si.torus(0.45, 0.15, rot=rot1), si.GridSpec((-0.8,) * 3, (20, 20, 20), 0.02)),
        "box_rot": (si.rounded_box((0.5, 0.35, 0.25), 0.06, rot=rot2), si.GridSpec((-0.9,) * 3, (18, 18, 18), 0.025)),
        "prism": (si.prism(si.PRISM_TRIANGLE, 0.0, 1.0), si.GridSpec((-0.2, -0.2, -0.2), (35, 30, 35), 0.01)),
        "torus_anisotropic": (si.torus(0.6, 0.2), si.GridSpec((-1.0, -1.0, -0.4), (50, 50, 20), 0.01)),
    }


CASES = _cases()


def build_both(sgm, name):
    shape, spec = CASES[name] if isinstance(name, str) else name
    g = sgm.Grid(spec)
    P = g.tag_allocate(shape)
    g.init_sdf(shape)
    O = oracle.build_grid(spec, shape)
    return g, O, P, shape, spec


# --------------------------------------------------------------------------
# A1 tagging / allocation, A2 init
# --------------------------------------------------------------------------
@pytest.mark.parametrize("name", list(CASES))
def test_tag_allocate_bit_exact(sg, name):
    g, O, P, shape, spec = build_both(sg, name)
    assert O.near_ties == 0
    assert P == O.P
    assert np.array_equal(H(g.field("cell_pkg")), O.cell_pkg)
    assert np.array_equal(H(g.field("pkg_cell")), O.pkg_cell)
    assert np.array_equal(H(g.field("pkg_type")), O.pkg_type)
    assert np.array_equal(H(g.field("nbr")), O.nbr)
    g.sync()


# Background grids whose rows, planes and total cell count fall across the
# 32-cell words of the tagging bit masks in every way: one-cell axes, rows of
# 31 and 33 cells, a plane of exactly 64 cells, and a count that is not a
# multiple of 32.
ODD_DIMS = [(1, 5, 7), (2, 33, 3), (31, 3, 17), (33, 1, 40), (8, 8, 9), (64, 1, 3), (7, 31, 1), (1, 1, 97)]


@pytest.mark.parametrize("dims", ODD_DIMS)
def test_tag_bit_mask_word_edges(sg, dims):
    h = 0.02
    lo = tuple(-2.0 * h * n for n in dims)  # the domain is centred on the origin
    spec = si.GridSpec(lo, dims, h)
    # a sphere through the middle of the box: core cells on every word edge
    shape = si.sphere(0.9 * 2.0 * h * max(min(dims), 2))
    g = sg.Grid(spec)
    P = g.tag_allocate(shape)
    cp, ct, P_o, ties = oracle.tag(spec, shape)
    assert ties == 0
    assert P == P_o
    assert np.array_equal(H(g.field("cell_pkg")), cp)
    pc, pt, nbr = oracle.tables(spec, cp, ct, P_o)
    assert np.array_equal(H(g.field("pkg_cell")), pc)
    assert np.array_equal(H(g.field("pkg_type")), pt)
    assert np.array_equal(H(g.field("nbr")), nbr)


@pytest.mark.parametrize("name", list(CASES))
def test_init_sdf_within_tolerance(sg, name):
    g, O, P, shape, spec = build_both(sg, name)
    phi = H(g.field("phi")).astype(np.float64)
    F = oracle.far_value(spec)
    assert np.all(phi[0] == np.float32(-F)) and np.all(phi[1] == np.float32(F))
    err = np.max(np.abs(phi[2:] - O.phi[2:]))
    assert err <= 1e-4 * spec.h, err
    # float-float evaluation rounds once: within one float32 ulp of the exact value
    assert np.all(np.abs(phi[2:] - O.phi[2:]) <= np.spacing(np.abs(O.phi[2:]).astype(np.float32)).astype(np.float64))


# --------------------------------------------------------------------------
# A3 gradient, Laplacian
# --------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["sphere_small", "torus_rot", "prism", "box_rot"])
def test_gradient_stepwise(sg, name):
    g, O, P, shape, spec = build_both(sg, name)
    g.gradient()
    phi = H(g.field("phi")).astype(np.float64)
    ref = oracle.gradient(spec, O.nbr, phi)
    for a, f in enumerate(("gx", "gy", "gz")):
        got = H(g.field(f)).astype(np.float64)
        assert np.max(np.abs(got - ref[a])) <= 1e-5
        assert np.all(got[:2] == 0)


@pytest.mark.parametrize("name", ["sphere_small", "torus_rot"])
def test_laplacian_stepwise(sg, name):
    g, O, P, shape, spec = build_both(sg, name)
    g.laplacian()
    phi = H(g.field("phi")).astype(np.float64)
    ref = oracle.laplacian(spec, O.nbr, phi)
    got = H(g.field("lap")).astype(np.float64)
    # float32 cancellation in phi(+) - 2 phi + phi(-): a few ulps of the
    # largest neighbour magnitude, divided by h^2
    tol = 8 * EPS32 * oracle.far_value(spec) / spec.h ** 2
    assert np.max(np.abs(got - ref)) <= tol


# --------------------------------------------------------------------------
# A4 reinitialisation
# --------------------------------------------------------------------------
def _distorted(spec, O, phi):
    nx, ny, nz = spec.dims
    pc = O.pkg_cell[2:].astype(np.int64)
    I, J, K = pc % nx, (pc // nx) % ny, pc // (nx * ny)
    d = np.arange(64)
    x = spec.lo[0] + (4 * I[:, None] + d % 4 + 0.5) * spec.h
    y = spec.lo[1] + (4 * J[:, None] + (d // 4) % 4 + 0.5) * spec.h
    z = spec.lo[2] + (4 * K[:, None] + d // 16 + 0.5) * spec.h
    out = phi.copy()
    out[2:] = phi[2:] * (0.5 + x * x + y * y + z * z)
    return out


@pytest.mark.parametrize("name", ["sphere_small", "torus_rot", "box_rot"])
@pytest.mark.parametrize("distort", [False, True])
def test_reinit_stepwise(sg, name, distort):
    shape, spec = CASES[name]
    O = oracle.build_grid(spec, shape)
    start = _distorted(spec, O, O.phi) if distort else O.phi
    start32 = start.astype(np.float32)
    states = []
    for k in (1, 2):
        g = sg.Grid(spec)
        g.tag_allocate(shape)
        g.init_sdf(shape)
        g.field("phi").copy_(torch.from_numpy(start32).cuda())
        g.reinit(k, 0.5)
        states.append(H(g.field("phi")).astype(np.float64))
    phi0 = start32.astype(np.float64)
    s0 = oracle.reinit_s0(spec, phi0)
    dt = 0.5 * spec.h
    ref1 = oracle.reinit_step(spec, O.nbr, phi0, s0, phi0, dt)
    ref2 = oracle.reinit_step(spec, O.nbr, phi0, s0, states[0], dt)
    assert np.max(np.abs(states[0] - ref1)) <= 1e-4 * spec.h
    assert np.max(np.abs(states[1] - ref2)) <= 1e-4 * spec.h
    assert np.array_equal(states[1][:2], start32[:2].astype(np.float64))


@pytest.mark.parametrize("name", ["sphere_small", "torus_rot"])
def test_reinit_smoothed_sign(sg, name):
    """S0 of a call: formed by its first sweep, or by a pass of its own when
    the call has no sweep; both the same floats, near the oracle's
    phi / sqrt(phi^2 + h^2), with -1 / +1 in the far packages."""
    shape, spec = CASES[name]
    O = oracle.build_grid(spec, shape)
    start32 = _distorted(spec, O, O.phi).astype(np.float32)
    got = []
    for iters in (0, 1, 4):
        g = sg.Grid(spec)
        g.tag_allocate(shape)
        g.init_sdf(shape)
        g.field("phi").copy_(torch.from_numpy(start32).cuda())
        g.reinit(iters, 0.5)
        got.append(H(g.field("S0")))
        g.sync()
    assert np.array_equal(got[0], got[1]) and np.array_equal(got[0], got[2])
    assert np.all(got[0][0] == -1.0) and np.all(got[0][1] == 1.0)
    ref = oracle.reinit_s0(spec, start32.astype(np.float64))
    assert np.max(np.abs(got[0][2:].astype(np.float64) - ref[2:])) <= 4 * EPS32


@pytest.mark.parametrize("iters", [20, 7])
def test_reinit_end_to_end_sphere_small(sg, iters):
    shape, spec = si.sphere_small()
    g = sg.Grid(spec)
    g.tag_allocate(shape)
    g.init_sdf(shape)
    O = oracle.build_grid(spec, shape)
    start = _distorted(spec, O, O.phi)
    g.field("phi").copy_(torch.from_numpy(start.astype(np.float32)).cuda())
    g.reinit(iters, 0.5)
    got = H(g.field("phi")).astype(np.float64)
    ref = oracle.reinit(spec, O.nbr, start.astype(np.float32).astype(np.float64), iters, 0.5)
    assert np.max(np.abs(got - ref)) <= 1e-4 * spec.h


# --------------------------------------------------------------------------
# A5 kernel integrals
# --------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["sphere_small", "torus_rot", "prism", "box_rot", "sphere_offset"])
def test_kernel_integrals_stepwise(sg, name):
    g, O, P, shape, spec = build_both(sg, name)
    g.kernel_integrals()
    phi = H(g.field("phi")).astype(np.float64)
    ref = oracle.kernel_integrals(spec, O.nbr, phi)
    for a, f in enumerate(("W", "Gx", "Gy", "Gz")):
        got = H(g.field(f)).astype(np.float64)
        assert np.max(np.abs(got - ref[a])) <= 1e-5, f
    W = H(g.field("W"))
    assert np.all(W[0] == 1) and np.all(W[1] == 0)


def test_kernel_integrals_plane_values(sg):
    """Plane through a data layer on a dyadic lattice: W = 1/2 at the layer."""
    h = 2.0 ** -5
    spec = si.GridSpec((-0.5, -0.5, -0.5), (8, 8, 8), h)
    z0 = spec.lo[2] + 15.5 * h
    shape = si.plane((0.0, 0.0, 1.0), point=(0.0, 0.0, z0))
    g = sg.Grid(spec)
    g.tag_allocate(shape)
    g.init_sdf(shape)
    g.kernel_integrals()
    O = oracle.build_grid(spec, shape)
    inner = (O.pkg_type >= 2) & np.all(O.nbr >= 2, axis=1)
    on = (O.phi == 0.0) & inner[:, None]
    W = H(g.field("W"))
    Gz = H(g.field("Gz"))
    assert on.sum() > 0
    assert np.max(np.abs(W[on] - 0.5)) <= 1e-6
    assert np.max(np.abs(Gz[on] + 0.475074612)) <= 1e-5


# --------------------------------------------------------------------------
# A6 probe and Morton order
# --------------------------------------------------------------------------
def _fields_host(g):
    return [H(g.field(f)).astype(np.float64) for f in ("phi", "gx", "gy", "gz", "W", "Gx", "Gy", "Gz")]


def _probe_compare(got, ref, h):
    assert np.max(np.abs(got["phi"] - ref[0])) <= 1e-4 * h
    for k, name in enumerate(("W", "Gx", "Gy", "Gz")):
        assert np.max(np.abs(got[name] - ref[4 + k])) <= 1e-5, name
    gref = np.sqrt(ref[1] ** 2 + ref[2] ** 2 + ref[3] ** 2)
    strong = gref > 0.5
    for k, name in enumerate(("nx", "ny", "nz")):
        assert np.max(np.abs(got[name][strong] - ref[1 + k][strong])) <= 1e-5, name


def test_probe_sphere_small(sg):
    """10,000 particles uniform within |phi| < 3h of the unit sphere (seed 0)."""
    shape, spec = si.sphere_small()
    g = sg.Grid(spec)
    g.tag_allocate(shape)
    g.init_sdf(shape)
    g.gradient()
    g.reinit(20, 0.5)
    g.gradient()
    g.kernel_integrals()
    x, y, z = si.sphere_shell_particles(10_000, 1.0, 3 * spec.h, seed=0)
    X, Y, Z = (torch.from_numpy(v).cuda() for v in (x, y, z))
    O = oracle.build_grid(spec, shape)
    fields = _fields_host(g)
    ref = oracle.probe(spec, O.cell_pkg, O.nbr, fields, x, y, z)
    for morton in (True, False):
        got = {k: H(v).astype(np.float64) for k, v in g.probe(X, Y, Z, morton=morton).items()}
        _probe_compare(got, ref, spec.h)


def test_probe_permutation_and_order_invariance(sg):
    shape, spec = CASES["torus_rot"]
    g = sg.Grid(spec)
    g.tag_allocate(shape)
    g.init_sdf(shape)
    g.gradient()
    g.kernel_integrals()
    x, y, z = si.box_particles(50_000, spec.lo, spec.hi(), seed=3)
    X, Y, Z = (torch.from_numpy(v).cuda() for v in (x, y, z))
    a = g.probe(X, Y, Z, morton=True)
    b = g.probe(X, Y, Z, morton=False)
    perm = torch.from_numpy(np.random.default_rng(0).permutation(len(x))).cuda()
    c = g.probe(X[perm], Y[perm], Z[perm], morton=True)
    for k in a:
        assert torch.equal(a[k], b[k])
        assert torch.equal(a[k][perm], c[k])
    O = oracle.build_grid(spec, shape)
    ref = oracle.probe(spec, O.cell_pkg, O.nbr, _fields_host(g), x, y, z)
    _probe_compare({k: H(v).astype(np.float64) for k, v in a.items()}, ref, spec.h)


def _keys_and_order_match(spec, x, y, z, keys, order):
    """Keys bit-exact against the oracle's definition (a particle within 1e-9
    of a lattice plane may carry either side's key: both decisions are
    correct there, and such particles must be rare), and the order the
    stable sort of those keys by (key, input index)."""
    k = H(keys).view(np.uint64)
    ok, n_tied = oracle.morton_keys_accept(spec, x, y, z, k)
    assert ok
    assert n_tied <= max(1, len(x) // 100_000)
    assert np.array_equal(H(order).astype(np.int64), oracle.morton_order(k))


@pytest.mark.parametrize("n", [1, 4095, 4096, 4097, 100_003])
def test_morton_order_bit_exact(sg, n):
    shape, spec = CASES["torus_anisotropic"]
    g = sg.Grid(spec)
    g.tag_allocate(shape)
    lo = np.array(spec.lo) - 0.1
    hi = np.array(spec.hi()) + 0.1
    x, y, z = si.box_particles(n, lo, hi, seed=n)
    # duplicates exercise the stability of equal keys
    if n > 10:
        x[n // 2:n // 2 + 5] = x[0]
        y[n // 2:n // 2 + 5] = y[0]
        z[n // 2:n // 2 + 5] = z[0]
    keys, order = g.morton_order(*(torch.from_numpy(v).cuda() for v in (x, y, z)))
    _keys_and_order_match(spec, x, y, z, keys, order)


def test_morton_sort_64bit_keys(sg):
    """Grids wide enough for keys over 32 bits take the 64-bit sort."""
    spec = si.GridSpec((-1.0, -1.0, -1.0), (600, 3, 3), 2.0 / 2400)
    shape = si.sphere(0.004)
    g = sg.Grid(spec)
    g.tag_allocate(shape)
    x, y, z = si.box_particles(20_000, spec.lo, spec.hi(), seed=9)
    keys, order = g.morton_order(*(torch.from_numpy(v).cuda() for v in (x, y, z)))
    assert int(oracle.morton_keys(spec, x, y, z).max()) >= 2 ** 32
    _keys_and_order_match(spec, x, y, z, keys, order)


# --------------------------------------------------------------------------
# Edge and degenerate cases, errors
# --------------------------------------------------------------------------
def test_empty_band_and_far_probe(sg):
    spec = si.GridSpec((-1.0,) * 3, (6, 6, 6), 0.05)
    for shape, inside in ((si.sphere(0.2, centre=(5.0, 5.0, 5.0)), False), (si.sphere(10.0), True)):
        g = sg.Grid(spec)
        assert g.tag_allocate(shape) == 2
        g.init_sdf(shape)
        g.gradient()
        g.reinit(3, 0.5)
        g.kernel_integrals()
        x, y, z = si.box_particles(1000, (-1.5,) * 3, (1.5,) * 3, seed=1)
        r = g.probe(*(torch.from_numpy(v).cuda() for v in (x, y, z)))
        cp = H(g.field("cell_pkg"))
        assert np.all(cp == (0 if inside else 1))
        F = 16 * spec.h
        # particles inside the domain see the far package of their cell
        inside_dom = np.all([(v >= spec.lo[a] + spec.h) & (v < spec.hi()[a] - spec.h) for a, v in
                             enumerate((x, y, z))], axis=0)
        assert np.allclose(H(r["phi"])[inside_dom], -F if inside else F, rtol=1e-6)
        assert np.all(H(r["nx"]) == 0)
        g.sync()


def test_probe_zero_particles(sg):
    shape, spec = si.sphere_small()
    g = sg.Grid(spec)
    g.tag_allocate(shape)
    g.init_sdf(shape)
    e = torch.empty(0, device="cuda")
    assert g.probe(e, e, e)["phi"].numel() == 0
    g.sync()


def test_retag_matches_fresh(sg):
    s1, spec = CASES["torus_rot"]
    s2 = si.sphere(0.5)
    g = sg.Grid(spec)
    g.tag_allocate(s1)
    g.init_sdf(s1)
    g.gradient()
    P2 = g.tag_allocate(s2)
    g.init_sdf(s2)
    O = oracle.build_grid(spec, s2)
    assert P2 == O.P
    assert np.array_equal(H(g.field("nbr")), O.nbr)
    assert np.max(np.abs(H(g.field("phi")).astype(np.float64) - O.phi)) <= 1e-4 * spec.h


@pytest.mark.parametrize("order", ["larger_first", "smaller_first"])
def test_retag_keeps_no_old_values(sg, order):
    """A re-tagged grid keeps its buffers but none of their values: fields not
    yet computed read as a fresh grid's (zeros, W = 1 / 0 in the far
    packages), and every computed field equals a fresh grid's bit for bit."""
    big, spec = CASES["torus_rot"]
    small = si.sphere(0.3)
    first, second = (big, small) if order == "larger_first" else (small, big)
    g = sg.Grid(spec)
    g.tag_allocate(first)
    g.init_sdf(first)
    g.gradient()
    g.reinit(3, 0.5)
    g.kernel_integrals()
    g.probe(*(torch.zeros(10, device="cuda") for _ in range(3)))
    g.tag_allocate(second)
    g.init_sdf(second)
    f = sg.Grid(spec)
    f.tag_allocate(second)
    f.init_sdf(second)
    for name in ("gx", "gy", "gz", "W", "Gx", "Gy", "Gz"):
        assert torch.equal(g.field(name), f.field(name)), name
    w = H(g.field("W"))
    assert np.all(w[0] == 1.0) and np.all(w[1] == 0.0) and np.all(w[2:] == 0.0)
    for grid in (g, f):
        grid.gradient()
        grid.reinit(3, 0.5)
        grid.kernel_integrals()
    for name in ("phi", "gx", "gy", "gz", "W", "Gx", "Gy", "Gz"):
        assert torch.equal(g.field(name), f.field(name)), name
    g.sync()
    f.sync()


def test_deterministic(sg):
    shape, spec = CASES["box_rot"]
    outs = []
    for _ in range(2):
        g = sg.Grid(spec)
        g.tag_allocate(shape)
        g.init_sdf(shape)
        g.reinit(5, 0.5)
        g.gradient()
        g.kernel_integrals()
        outs.append([g.field(f).clone() for f in ("phi", "gx", "W", "Gz")])
    for a, b in zip(*outs):
        assert torch.equal(a, b)


def test_error_codes(sg):
    shape, spec = si.sphere_small()
    g = sg.Grid(spec)
    with pytest.raises(sg.SgError) as e:
        g.gradient()
    assert e.value.status == sg.SG_ERR_STATE
    with pytest.raises(sg.SgError) as e:
        g.init_sdf(shape)
    assert e.value.status == sg.SG_ERR_STATE
    g.tag_allocate(shape)
    with pytest.raises(sg.SgError) as e:
        g.reinit(5, 0.5)
    assert e.value.status == sg.SG_ERR_STATE
    g.init_sdf(shape)
    with pytest.raises(sg.SgError) as e:
        g.reinit(5, -1.0)
    assert e.value.status == sg.SG_ERR_INVALID
    with pytest.raises(sg.SgError) as e:
        g.reinit(-1, 0.5)
    assert e.value.status == sg.SG_ERR_INVALID
    with pytest.raises(sg.SgError) as e:
        g.kernel_integrals(mode=7)
    assert e.value.status == sg.SG_ERR_INVALID
    bad = si.Shape(9)
    with pytest.raises(sg.SgError) as e:
        g.tag_allocate(bad)
    assert e.value.status == sg.SG_ERR_INVALID
    with pytest.raises(sg.SgError) as e:
        sg.Grid(si.GridSpec((0, 0, 0), (600000, 1, 1), 0.1))
    assert e.value.status == sg.SG_ERR_CAPACITY
    with pytest.raises(sg.SgError) as e:
        sg.Grid(si.GridSpec((0, 0, 0), (0, 1, 1), 0.1))
    assert e.value.status == sg.SG_ERR_INVALID
    g.sync()  # the grid is still usable after rejected calls
    g.gradient()
    g.sync()


def test_allocator_hook_and_default_pool(sg):
    shape, spec = CASES["sphere_offset"]
    a = sg.Grid(spec, torch_allocator=True)
    b = sg.Grid(spec, torch_allocator=False)
    for g in (a, b):
        g.tag_allocate(shape)
        g.init_sdf(shape)
        g.gradient()
    assert torch.equal(a.field("gx"), b.field("gx"))
    a.close()
    b.close()


def test_morton_sorted_input_fast_path(sg):
    """Keys already in order: identity order, same keys; one swapped pair
    forces the full sort; probe results do not depend on the path."""
    shape, spec = CASES["torus_anisotropic"]
    g = sg.Grid(spec)
    g.tag_allocate(shape)
    g.init_sdf(shape)
    g.gradient()
    g.kernel_integrals()
    x, y, z = si.box_particles(100_000, spec.lo, spec.hi(), seed=77)
    rk = oracle.morton_keys(spec, x, y, z)
    ro = oracle.morton_order(rk)
    xs, ys, zs = x[ro], y[ro], z[ro]
    D = [torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (xs, ys, zs)]
    keys, order = g.morton_order(*D)
    assert np.array_equal(H(order), np.arange(len(xs)))
    assert oracle.lattice_ties(spec, xs, ys, zs) == 0  # the input order was the oracle's
    assert np.array_equal(H(keys).view(np.uint64), rk[ro])
    a = g.probe(*D, morton=True)
    b = g.probe(*D, morton=False)
    for k in a:
        assert torch.equal(a[k], b[k])
    # swap two particles with different keys: no longer sorted
    i, j = 10, 50_000
    assert rk[ro[i]] != rk[ro[j]]
    xs2, ys2, zs2 = xs.copy(), ys.copy(), zs.copy()
    for v in (xs2, ys2, zs2):
        v[i], v[j] = v[j], v[i]
    D2 = [torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (xs2, ys2, zs2)]
    keys2, order2 = g.morton_order(*D2)
    _keys_and_order_match(spec, xs2, ys2, zs2, keys2, order2)
    c = g.probe(*D2, morton=True)
    d = g.probe(*D2, morton=False)
    for k in c:
        assert torch.equal(c[k], d[k])
