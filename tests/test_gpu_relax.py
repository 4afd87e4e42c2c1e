"""Batched surrogate integrals and batched particle relaxation on the GPU.

* integrals_mode 1 in a batch equals the single-grid surrogate per body, bit
  for bit;
* relaxation, step-wise: from the same float32 start and the same fields
  (the batch's, widened), one step lands within one float32 rounding of the
  oracle's step (the displacement itself differs by ~1e-7 h) and the probe
  outputs meet the probe tolerances; K steps stay within K roundings;
* end to end against the oracle's own chain (init, gradient, 20 reinit
  sweeps, integrals): the fields differ by at most 1e-4 h in phi and 1e-5 in
  g, which moves a particle by at most 1.2e-5 h per step, so K steps stay
  within K (2e-5 h + 1 ulp);
* graph replays continue the relaxation exactly; empty bodies are skipped;
* at full size (64 mixed bodies, 10^8 particles, 50 steps, surrogate
  integrals) on a sample of particles.
"""
import numpy as np
import pytest

import oracle
import sg_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ("phi", "gx", "gy", "gz", "W", "Gx", "Gy", "Gz")
OUTS = ("phi", "nx", "ny", "nz", "W", "Gx", "Gy", "Gz")


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


def _grids(sg, bodies):
    gs = []
    for shape, spec, _ in bodies:
        g = sg.Grid(spec)
        g.tag_allocate(shape)
        g.init_sdf(shape)
        gs.append(g)
    return gs


def _sorted_particles(sg, grids, x, y, z, off):
    """Device particles, each body's segment in its Morton order."""
    X = [torch.from_numpy(v).cuda() for v in (x, y, z)]
    for b, g in enumerate(grids):
        s, e = int(off[b]), int(off[b + 1])
        if e == s:
            continue
        seg = [v[s:e] for v in X]
        _, order = g.morton_order(*seg)
        o = order.long()
        for v, sv in zip(X, seg):
            v[s:e] = sv[o]
    return X


def _ulp(v):
    return np.spacing(np.abs(np.asarray(v, np.float32))).astype(np.float64)


def _body_fields(batch, b):
    return [H(batch.field(b, f)).astype(np.float64) for f in FIELDS]


@pytest.fixture(scope="module")
def small(sg):
    bodies = si.random_bodies(6, seed=1, p_lo=1e2, p_hi=3e3)
    grids = _grids(sg, bodies)
    x, y, z, off = si.relax_particles(bodies, 120_000, seed=5)
    X = _sorted_particles(sg, grids, x, y, z, off)
    O = [oracle.build_grid(spec, shape) for shape, spec, _ in bodies]
    for g, o in zip(grids, O):
        assert np.array_equal(H(g.field("cell_pkg")), o.cell_pkg)
        assert np.array_equal(H(g.field("nbr")), o.nbr)
    return bodies, grids, X, off, O


def _relax(sg, batch, X, off, steps, sweeps, plan=None, outs=OUTS):
    Y = [v.clone() for v in X]
    out = {k: torch.full_like(Y[0], float("nan")) for k in outs}
    batch.relax(*Y, off, steps, 0.1, plan=plan, sweeps=sweeps, out=out)
    torch.cuda.synchronize()
    return Y, out


def test_batch_surrogate_equals_single_grid(sg, small):
    bodies, grids, _, _, _ = small
    net = sg.MLP(si.mlp_init_params(seed=4))
    ref = []
    for g in _grids(sg, bodies):
        g.gradient()
        g.reinit(20, 0.5)
        g.kernel_integrals(mode=1, mlp=net)
        ref.append({f: g.field(f).clone() for f in FIELDS})
    batch = sg.Batch(grids)
    with pytest.raises(sg.SgError):  # mode 1 needs a bound network
        batch.run(sg.make_plan(4, 2, 20, 0.5, integrals_mode=1))
    batch.set_surrogate(net)
    for ppi, depth in ((8, 1), (2, 2)):
        batch.reset()
        batch.run(sg.make_plan(ppi, depth, 20, 0.5, integrals_mode=1))
        for b, r in enumerate(ref):
            for f in FIELDS:
                assert torch.equal(batch.field(b, f), r[f]), (ppi, b, f)
    batch.close()
    net.close()


def _check_positions(bodies, off, Y, ref_xyz, K, b_list=None):
    for b, (shape, spec, _) in enumerate(bodies):
        s, e = int(off[b]), int(off[b + 1])
        for a in range(3):
            got = H(Y[a][s:e]).astype(np.float64)
            want = ref_xyz[b][a].astype(np.float64)
            tol = K * (_ulp(want) + 1e-6 * spec.h)
            assert np.all(np.abs(got - want) <= tol), (b, a, np.max(np.abs(got - want) / tol))


def test_relax_one_step_matches_oracle(sg, small):
    bodies, grids, X, off, O = small
    batch = sg.Batch(grids)
    plan = sg.make_plan(4, 2, 20, 0.5)
    Y, out = _relax(sg, batch, X, off, 1, True, plan)
    ref_xyz = []
    for b, (shape, spec, _) in enumerate(bodies):
        s, e = int(off[b]), int(off[b + 1])
        x0 = [H(v[s:e]) for v in X]
        fields = _body_fields(batch, b)
        xyz, ro = oracle.relax(spec, O[b].cell_pkg, O[b].nbr, fields, *x0, 1, 0.1)
        ref_xyz.append(xyz)
        got = {k: H(out[k][s:e]).astype(np.float64) for k in OUTS}
        assert np.max(np.abs(got["phi"] - ro[0])) <= 1e-4 * spec.h
        for k in range(4, 8):
            assert np.max(np.abs(got[OUTS[k]] - ro[k])) <= 1e-5
        # n is compared where the interpolated gradient is strong (|g| > 0.5):
        # the gradient rides in the integral slots of a second probe
        gf = fields[:4] + fields[1:4] + [fields[0]]
        gi = oracle.probe(spec, O[b].cell_pkg, O[b].nbr, gf, *x0)
        strong = np.sqrt(gi[4] ** 2 + gi[5] ** 2 + gi[6] ** 2) > 0.5
        assert strong.mean() > 0.5
        for k in range(1, 4):
            assert np.max(np.abs(got[OUTS[k]][strong] - ro[k][strong])) <= 1e-5
    _check_positions(bodies, off, Y, ref_xyz, 1)
    batch.close()


def test_relax_k_steps_same_fields(sg, small):
    bodies, grids, X, off, O = small
    batch = sg.Batch(grids)
    plan = sg.make_plan(8, 1, 20, 0.5)
    K = 12
    Y, _ = _relax(sg, batch, X, off, K, True, plan, outs=())
    ref_xyz = []
    for b, (shape, spec, _) in enumerate(bodies):
        s, e = int(off[b]), int(off[b + 1])
        xyz, _ = oracle.relax(spec, O[b].cell_pkg, O[b].nbr, _body_fields(batch, b), *[H(v[s:e]) for v in X], K, 0.1)
        ref_xyz.append(xyz)
    _check_positions(bodies, off, Y, ref_xyz, K)
    batch.close()


def test_relax_end_to_end_oracle_chain(sg, small):
    bodies, grids, X, off, O = small
    batch = sg.Batch(grids)
    K = 5
    Y, _ = _relax(sg, batch, X, off, K, True, sg.make_plan(4, 1, 20, 0.5), outs=())
    for b, (shape, spec, _) in enumerate(bodies):
        s, e = int(off[b]), int(off[b + 1])
        g = oracle.gradient(spec, O[b].nbr, O[b].phi)
        phi = oracle.reinit(spec, O[b].nbr, O[b].phi, 20, 0.5)
        wi = oracle.kernel_integrals(spec, O[b].nbr, phi)
        fields = (phi, g[0], g[1], g[2], wi[0], wi[1], wi[2], wi[3])
        xyz, _ = oracle.relax(spec, O[b].cell_pkg, O[b].nbr, fields, *[H(v[s:e]) for v in X], K, 0.1)
        for a in range(3):
            got = H(Y[a][s:e]).astype(np.float64)
            want = xyz[a].astype(np.float64)
            assert np.all(np.abs(got - want) <= K * (2e-5 * spec.h + _ulp(want))), (b, a)
    batch.close()


def test_relax_steps_beyond_one_launch(sg, small):
    """A call runs at most 64 steps per launch: 70 steps in one call (64 + 6)
    equal seven calls of 10 steps bit for bit, positions and outputs."""
    bodies, grids, X, off, O = small
    batch = sg.Batch(grids)
    plan = sg.make_plan(4, 1, 20, 0.5)
    Y70, o70 = _relax(sg, batch, X, off, 70, True, plan)
    batch.reset()
    batch.run(plan)
    Y = [v.clone() for v in X]
    out = {k: torch.empty_like(Y[0]) for k in OUTS}
    for _ in range(7):
        batch.relax(*Y, off, 10, 0.1, sweeps=False, out=out)
    torch.cuda.synchronize()
    for a in range(3):
        assert torch.equal(Y[a], Y70[a])
    for k in OUTS:
        assert torch.equal(out[k], o70[k])
    assert max(float((a - b).abs().max()) for a, b in zip(Y70, X)) > 0  # the particles moved
    batch.close()


def test_relax_replay_sweeps_and_empty_bodies(sg, small):
    bodies, grids, X, off, O = small
    batch = sg.Batch(grids)
    plan = sg.make_plan(4, 2, 20, 0.5)
    # 6 steps at once
    Y6, o6 = _relax(sg, batch, X, off, 6, True, plan)
    # the same fields (sweeps recomputed from the reset phi), 3 + 3 steps by replaying one graph
    batch.reset()
    batch.run(plan)
    Y = [v.clone() for v in X]
    out = {k: torch.empty_like(Y[0]) for k in OUTS}
    for _ in range(2):
        batch.relax(*Y, off, 3, 0.1, sweeps=False, out=out)
    torch.cuda.synchronize()
    for a in range(3):
        assert torch.equal(Y[a], Y6[a])
    for k in OUTS:
        assert torch.equal(out[k], o6[k])
    # and six calls of one step each: a launch per step, against one launch
    # that takes every particle through the six steps
    batch.reset()
    batch.run(plan)
    Z = [v.clone() for v in X]
    for _ in range(6):
        batch.relax(*Z, off, 1, 0.1, sweeps=False, out=out)
    torch.cuda.synchronize()
    for a in range(3):
        assert torch.equal(Z[a], Y6[a])
    for k in OUTS:
        assert torch.equal(out[k], o6[k])
    # bodies 1 and 5 without particles: the others move exactly as before
    keep = [b for b in range(len(bodies)) if b not in (1, 5)]
    segs = [(int(off[b]), int(off[b + 1])) for b in keep]
    sub = [torch.cat([v[s:e] for s, e in segs]) for v in X]
    cnt = np.zeros(len(bodies) + 1, np.int64)
    for b in keep:
        cnt[b + 1] = off[b + 1] - off[b]
    off2 = np.cumsum(cnt)
    Z = [v.clone() for v in sub]
    batch.relax(*Z, off2, 6, 0.1, sweeps=False)
    torch.cuda.synchronize()
    want = [torch.cat([v[s:e] for s, e in segs]) for v in Y6]
    for a in range(3):
        assert torch.equal(Z[a], want[a])
    # malformed offsets are refused before any launch
    bad = off.copy()
    bad[2] = bad[3] + 1
    with pytest.raises(sg.SgError):
        batch.relax(*Z, bad, 1, 0.1, sweeps=False)
    batch.close()


N_FULL = 100_000_000


def test_relax_full_size_sampled(sg):
    """The relaxation workload as bench.py runs it: the first 64 bodies of the
    256-body batch, 10^8 particles, sweeps with surrogate integrals, 50 steps;
    49 steps are compared on a sample against the oracle from the same start
    and fields, and the 50th step-wise with its probe outputs."""
    bodies = si.random_bodies(64, seed=1)
    grids = _grids(sg, bodies)
    x, y, z, off = si.relax_particles(bodies, N_FULL, seed=5)
    X = _sorted_particles(sg, grids, x, y, z, off)
    del x, y, z
    net = sg.MLP(si.mlp_init_params(seed=4))
    batch = sg.Batch(grids)
    batch.set_surrogate(net)
    plan = sg.make_plan(8, 1, 20, 0.5, integrals_mode=1)
    rng = np.random.default_rng(3)
    sample = np.sort(rng.choice(N_FULL, 200_000, replace=False))
    st = torch.from_numpy(sample).cuda()
    x0 = [H(v[st]) for v in X]
    batch.relax(*X, off, 49, 0.1, plan=plan, sweeps=True)
    torch.cuda.synchronize()
    x49 = [H(v[st]) for v in X]
    out = {k: torch.empty_like(X[0]) for k in OUTS}
    batch.relax(*X, off, 1, 0.1, sweeps=False, out=out)
    torch.cuda.synchronize()
    x50 = [H(v[st]) for v in X]
    got = {k: H(out[k][st]).astype(np.float64) for k in OUTS}
    body_of = np.searchsorted(off, sample, side="right") - 1
    for b, (shape, spec, _) in enumerate(bodies):
        m = body_of == b
        if not m.any():
            continue
        O = oracle.build_grid(spec, shape)
        assert np.array_equal(H(batch.field(b, "cell_pkg")) - batch_base(batch, b), O.cell_pkg)
        fields = _body_fields(batch, b)
        xyz, _ = oracle.relax(spec, O.cell_pkg, O.nbr, fields, *[v[m] for v in x0], 49, 0.1)
        for a in range(3):
            want = xyz[a].astype(np.float64)
            assert np.all(np.abs(x49[a][m] - want) <= 49 * (_ulp(want) + 1e-6 * spec.h)), (b, a)
        xyz, ro = oracle.relax(spec, O.cell_pkg, O.nbr, fields, *[v[m] for v in x49], 1, 0.1)
        for a in range(3):
            want = xyz[a].astype(np.float64)
            assert np.all(np.abs(x50[a][m] - want) <= _ulp(want) + 1e-6 * spec.h), (b, a)
        assert np.max(np.abs(got["phi"][m] - ro[0])) <= 1e-4 * spec.h
        for k in range(4, 8):
            assert np.max(np.abs(got[OUTS[k]][m] - ro[k])) <= 1e-5, (b, OUTS[k])
    batch.close()
    net.close()


def batch_base(batch, b):
    """Global id of body b's first package (its far- package)."""
    return int(H(batch.field(b, "nbr"))[0, 0])
