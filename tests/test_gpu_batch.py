"""Batched sweeps over many bodies against the single-grid calls.

A batch concatenates the bodies' packages into one store and runs each sweep
as one persistent launch; per body the results must equal the single-grid
gradient -> reinit -> integrals chain bit for bit, for every schedule, on
graph replays and for odd sweep counts.
"""
import numpy as np
import pytest

import sg_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ("phi", "gx", "gy", "gz", "W", "Gx", "Gy", "Gz")


@pytest.fixture(scope="module")
def sg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11473_b300 import build
    build.build()
    import paper_2512_11473_b300 as m
    return m


def _bodies():
    out = [(s, g) for s, g, _ in si.random_bodies(7, seed=1, p_lo=1e2, p_hi=4e3)]
    out.append(si.sphere_small())
    return out


def _grids(sg, bodies):
    gs = []
    for shape, spec in bodies:
        g = sg.Grid(spec)
        g.tag_allocate(shape)
        g.init_sdf(shape)
        gs.append(g)
    return gs


def _single(sg, bodies, iters, cfl=0.5):
    ref = []
    for g in _grids(sg, bodies):
        g.gradient()
        g.reinit(iters, cfl)
        g.kernel_integrals()
        ref.append({f: g.field(f).clone() for f in FIELDS})
    return ref


@pytest.fixture(scope="module")
def setup(sg):
    bodies = _bodies()
    return bodies, _grids(sg, bodies), _single(sg, bodies, 20), _single(sg, bodies, 7)


def _check(batch, ref):
    for b, r in enumerate(ref):
        for f in FIELDS:
            assert torch.equal(batch.field(b, f), r[f]), (b, f)


@pytest.mark.parametrize("ppi,depth", [(1, 1), (2, 2), (4, 1), (8, 2)])
def test_batch_equals_single_grid(sg, setup, ppi, depth):
    bodies, grids, ref20, _ = setup
    batch = sg.Batch(grids)
    assert batch.P == sum(g.P for g in grids)
    batch.run(pkgs_per_item=ppi, depth=depth, reinit_iterations=20, cfl=0.5)
    _check(batch, ref20)
    batch.close()


def test_batch_replay_and_odd_sweeps(sg, setup):
    bodies, grids, ref20, ref7 = setup
    batch = sg.Batch(grids)
    plan = sg.make_plan(4, 2, 7, 0.5)
    batch.run(plan)
    _check(batch, ref7)
    for _ in range(2):  # replays of the captured graph start from the reset phi
        batch.reset()
        batch.run(plan)
        _check(batch, ref7)
    batch.reset()
    batch.run(pkgs_per_item=2, depth=1, reinit_iterations=20)
    _check(batch, ref20)
    torch.cuda.synchronize()


def test_batch_autotune(sg, setup):
    bodies, grids, ref20, _ = setup
    batch = sg.Batch(grids)
    plan, times = batch.autotune(sg.make_plan(reinit_iterations=20), reps=2)
    assert (plan.pkgs_per_item, plan.depth) in times
    assert all(np.isfinite(v) and v > 0 for v in times.values())
    assert times[(plan.pkgs_per_item, plan.depth)] == min(times.values())
    batch.run(plan)
    _check(batch, ref20)


def test_batch_autotune_cached(sg, setup, tmp_path):
    """The first call tunes and appends its choice to the cache file; the
    second finds it there (no runs) and returns the same plan."""
    bodies, grids, ref20, _ = setup
    batch = sg.Batch(grids)
    path = tmp_path / "tune.txt"
    key = batch.autotune_key(sg.make_plan(reinit_iterations=20))
    assert key.startswith("gpu=") and ";sweeps=20;integrals=0;packages=2^" in key and " " not in key
    p1, hit1 = batch.autotune_cached(path, sg.make_plan(reinit_iterations=20), reps=2)
    assert not hit1
    assert (p1.pkgs_per_item, p1.depth) in sg.BATCH_CANDIDATES
    assert path.read_text().splitlines() == ["%s %d %d" % (key, p1.pkgs_per_item, p1.depth)]
    assert sg.autotune_cache_lookup(path, key) == (p1.pkgs_per_item, p1.depth)
    p2, hit2 = batch.autotune_cached(path, sg.make_plan(reinit_iterations=20), reps=2)
    assert hit2 and (p2.pkgs_per_item, p2.depth) == (p1.pkgs_per_item, p1.depth)
    assert len(path.read_text().splitlines()) == 1
    # another sweep count is another key: tuned and appended
    p3, hit3 = batch.autotune_cached(path, sg.make_plan(reinit_iterations=7), reps=1)
    assert not hit3 and len(path.read_text().splitlines()) == 2
    batch.run(p2)
    _check(batch, ref20)


def test_batch_global_neighbour_ids(sg, setup):
    bodies, grids, _, _ = setup
    batch = sg.Batch(grids)
    base = 0
    for b, g in enumerate(grids):
        assert torch.equal(batch.field(b, "nbr"), g.field("nbr") + base)
        base += g.P


def test_batch_errors(sg, setup):
    bodies, grids, _, _ = setup
    batch = sg.Batch(grids)
    with pytest.raises(sg.SgError) as e:
        batch.run(pkgs_per_item=3)
    assert e.value.status == sg.SG_ERR_INVALID
    with pytest.raises(sg.SgError) as e:
        batch.run(pkgs_per_item=1, depth=2)
    assert e.value.status == sg.SG_ERR_INVALID
    g = sg.Grid(bodies[0][1])
    g.tag_allocate(bodies[0][0])
    with pytest.raises(sg.SgError) as e:
        sg.Batch([g])
    assert e.value.status == sg.SG_ERR_STATE
