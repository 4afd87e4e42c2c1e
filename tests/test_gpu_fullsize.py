"""Parity at full size: the torus and the prism at h = 0.002 (362,290 and
254,701 packages), as bench.py runs them.

Whole arrays are compared where the oracle finishes in seconds (tags, phi,
gradient, 50 reinit sweeps, kernel integrals); the 50M-particle probe is
checked on a 1M-particle sample of its outputs (the oracle probes particles
one by one) and by invariants of the Morton order at full size.
"""
import numpy as np
import pytest

import oracle
import sg_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_PARTICLES = 50_000_000


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


@pytest.fixture(scope="module", params=["torus", "prism"])
def body(request, sg):
    name = request.param
    shape, spec = si.torus_large() if name == "torus" else si.prism_large()
    g = sg.Grid(spec)
    P = g.tag_allocate(shape)
    g.init_sdf(shape)
    O = oracle.build_grid(spec, shape)
    return name, shape, spec, g, P, O


def test_full_tags_and_phi(body):
    name, shape, spec, g, P, O = body
    assert O.near_ties == 0
    assert P == O.P
    assert np.array_equal(H(g.field("cell_pkg")), O.cell_pkg)
    assert np.array_equal(H(g.field("pkg_type")), O.pkg_type)
    assert np.array_equal(H(g.field("pkg_cell")), O.pkg_cell)
    assert np.array_equal(H(g.field("nbr")), O.nbr)
    phi = H(g.field("phi")).astype(np.float64)
    assert np.max(np.abs(phi - O.phi)) <= 1e-4 * spec.h


def test_full_gradient_reinit_integrals(body, sg):
    name, shape, spec, g, P, O = body
    g.init_sdf(shape)
    phi0 = H(g.field("phi")).astype(np.float64)
    g.gradient()
    ref = oracle.gradient(spec, O.nbr, phi0)
    for a, f in enumerate(("gx", "gy", "gz")):
        assert np.max(np.abs(H(g.field(f)) - ref[a])) <= 1e-5
    # 50 sweeps end to end, both chains from the device's initial phi
    g.reinit(50, 0.5)
    phi = H(g.field("phi")).astype(np.float64)
    ref_phi = oracle.reinit(spec, O.nbr, phi0, 50, 0.5)
    assert np.max(np.abs(phi - ref_phi)) <= 1e-4 * spec.h
    g.kernel_integrals()
    ref = oracle.kernel_integrals(spec, O.nbr, phi)
    for a, f in enumerate(("W", "Gx", "Gy", "Gz")):
        assert np.max(np.abs(H(g.field(f)) - ref[a])) <= 1e-5


def test_full_probe_50m_sampled(body, sg):
    """The bench configuration: 50M band particles (+-2 coarse cells, +-0.5h
    jitter), stored in Morton order, probed with SG_PROBE_MORTON."""
    import bench
    name, shape, spec, g, P, O = body
    x, y, z = bench.particles_for(name, shape, spec, N_PARTICLES, 2 if name == "torus" else 3)
    dev = [torch.from_numpy(v).cuda() for v in (x, y, z)]
    keys, order = g.morton_order(*dev)
    # Morton order at full size: a permutation, keys non-decreasing, ties by index
    o = order.long()
    k_sorted = keys[o]
    assert bool((k_sorted[1:] >= k_sorted[:-1]).all())
    tie = k_sorted[1:] == k_sorted[:-1]
    assert bool((o[1:][tie] > o[:-1][tie]).all())
    seen = torch.zeros(N_PARTICLES, dtype=torch.int32, device="cuda")
    seen.index_add_(0, o, torch.ones_like(order))
    assert bool((seen == 1).all())
    del seen, tie, k_sorted
    X = [v[o].contiguous() for v in dev]
    del dev
    g.init_sdf(shape)
    g.gradient()
    g.reinit(50, 0.5)
    g.kernel_integrals()
    out = g.probe(*X, morton=True)
    rng = np.random.default_rng(7)
    sample = np.sort(rng.choice(N_PARTICLES, 1_000_000, replace=False))
    si_t = torch.from_numpy(sample).cuda()
    xs, ys, zs = (H(v[si_t]) for v in X)
    # keys of the sample against the oracle's definition (a particle within
    # 1e-9 of a lattice plane may carry either side's key)
    ok, n_tied = oracle.morton_keys_accept(spec, xs, ys, zs, H(keys[o[si_t]]))
    assert ok and n_tied <= 10
    fields = [H(g.field(f)).astype(np.float64) for f in ("phi", "gx", "gy", "gz", "W", "Gx", "Gy", "Gz")]
    ref = oracle.probe(spec, O.cell_pkg, O.nbr, fields, xs, ys, zs)
    got = {k: H(v[si_t]).astype(np.float64) for k, v in out.items()}
    assert np.max(np.abs(got["phi"] - ref[0])) <= 1e-4 * spec.h
    for k, name_ in enumerate(("W", "Gx", "Gy", "Gz")):
        assert np.max(np.abs(got[name_] - ref[4 + k])) <= 1e-5
    gref = np.sqrt(ref[1] ** 2 + ref[2] ** 2 + ref[3] ** 2)
    strong = gref > 0.5
    for k, name_ in enumerate(("nx", "ny", "nz")):
        assert np.max(np.abs(got[name_][strong] - ref[1 + k][strong])) <= 1e-5
    g.sync()


def test_full_surrogate_classes(body, sg):
    """Surrogate integrals at full size (random weights: the classes and the
    fallback do not depend on them): pass A's class counts equal the
    classification kernel's, the classes equal the oracle's FP64 definition
    with no point within 1e-9 of a threshold, fallback points carry the
    exact sums bit for bit and trivial points the exact constants."""
    name, shape, spec, g, P, O = body
    g.init_sdf(shape)
    g.reinit(50, 0.5)
    g.kernel_integrals()
    exact = {f: g.field(f).clone() for f in ("W", "Gx", "Gy", "Gz")}
    net = sg.MLP(si.mlp_init_params(16))
    g.kernel_integrals(mode=1, mlp=net)
    cls = g.surrogate_classify()
    assert g.surrogate_stats() == [int((cls[2:] == c).sum()) for c in range(4)]
    ref, ties = oracle.surrogate_class(spec, O.nbr, H(g.field("phi")), ties=True)
    assert ties == 0
    assert np.array_equal(H(cls), ref)
    fb = cls == 2
    for f in exact:
        assert torch.equal(g.field(f)[fb], exact[f][fb]), f
    tin, tout = cls == 0, cls == 1
    assert bool((g.field("W")[tin] == 1).all()) and bool((g.field("W")[tout] == 0).all())
    for f in ("Gx", "Gy", "Gz"):
        assert bool((g.field(f)[tin | tout] == 0).all()), f
    net.close()
