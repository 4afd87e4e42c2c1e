"""Batched sweeps against the FP64 oracle, body by body.

Seven bodies of very different package counts (six random bodies and the
small sphere) run as one batch under two schedules, with exact and with
surrogate integrals.  Each body's fields are compared element by element
with the oracle on that body's own tables:

* gradient of the initial phi (step-wise, <= 1e-5);
* phi after 20 Jacobi reinit sweeps from the same initial phi (end to end,
  <= 1e-4 h);
* kernel integrals W, G^ of the batch's final phi (step-wise, <= 1e-5);
* surrogate mode: classes against the oracle's decision on the batch's phi,
  trivial points exactly (1, 0) / (0, 0), fallback points bit for bit equal
  to the exact-mode batch values, network points against the oracle network
  on the oracle's canonical inputs (<= 2e-2 of the output scale, the BF16
  activations' bar of the single-grid test).
"""
import numpy as np
import pytest

import oracle
import sg_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CFL = 0.5
ITERS = 20


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


def bf16_round(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


@pytest.fixture(scope="module")
def setup(sg):
    bodies = [(s, g) for s, g, _ in si.random_bodies(6, seed=3, p_lo=1e2, p_hi=3e3)]
    bodies.append(si.sphere_small())
    grids, ref = [], []
    for shape, spec in bodies:
        g = sg.Grid(spec)
        g.tag_allocate(shape)
        g.init_sdf(shape)
        grids.append(g)
        O = oracle.build_grid(spec, shape)
        phi0 = H(g.field("phi")).astype(np.float64)
        ref.append({"spec": spec, "O": O, "phi0": phi0,
                    "g": oracle.gradient(spec, O.nbr, phi0),
                    "phi": oracle.reinit(spec, O.nbr, phi0, ITERS, CFL)})
    return bodies, grids, ref


@pytest.mark.parametrize("ppi,depth", [(2, 1), (8, 2)])
def test_batch_exact_against_oracle(sg, setup, ppi, depth):
    bodies, grids, ref = setup
    batch = sg.Batch(grids)
    batch.run(pkgs_per_item=ppi, depth=depth, reinit_iterations=ITERS, cfl=CFL)
    for b, r in enumerate(ref):
        spec, O = r["spec"], r["O"]
        assert np.array_equal(H(batch.field(b, "nbr")) - H(batch.field(b, "nbr"))[0, 0], O.nbr)  # far- package is its own neighbour
        for a, f in enumerate(("gx", "gy", "gz")):
            assert np.max(np.abs(H(batch.field(b, f)) - r["g"][a])) <= 1e-5, (b, f)
        phi = H(batch.field(b, "phi")).astype(np.float64)
        assert np.max(np.abs(phi - r["phi"])) <= 1e-4 * spec.h, b
        integ = oracle.kernel_integrals(spec, O.nbr, phi)
        for a, f in enumerate(("W", "Gx", "Gy", "Gz")):
            assert np.max(np.abs(H(batch.field(b, f)) - integ[a])) <= 1e-5, (b, f)
    batch.close()


@pytest.mark.parametrize("ppi,depth", [(4, 1), (1, 1)])
def test_batch_surrogate_against_oracle(sg, setup, ppi, depth):
    bodies, grids, ref = setup
    par = si.mlp_init_params(16)
    net = sg.MLP(par)
    exact = sg.Batch(grids)
    exact.run(pkgs_per_item=ppi, depth=depth, reinit_iterations=ITERS, cfl=CFL)
    batch = sg.Batch(grids)
    batch.set_surrogate(net)
    batch.run(sg.make_plan(ppi, depth, ITERS, CFL, integrals_mode=1))
    n_net = 0
    for b, r in enumerate(ref):
        spec, O = r["spec"], r["O"]
        phi32 = H(batch.field(b, "phi"))
        assert np.array_equal(phi32, H(exact.field(b, "phi")))
        cls, ties = oracle.surrogate_class(spec, O.nbr, phi32, ties=True)
        assert ties == 0
        got = np.stack([H(batch.field(b, f)) for f in ("W", "Gx", "Gy", "Gz")], -1)
        ex = np.stack([H(exact.field(b, f)) for f in ("W", "Gx", "Gy", "Gz")], -1)
        fb, net_pts = cls == 2, cls == 3
        assert np.array_equal(got[fb], ex[fb]), b
        assert np.all(got[cls == 0] == [1.0, 0.0, 0.0, 0.0]) and np.all(got[cls == 1] == 0.0)
        if net_pts.any():
            xin, code = oracle.surrogate_canonical(spec, O.nbr, phi32)
            y = oracle.mlp_forward(bf16_round(par), bf16_round(xin[net_pts].astype(np.float32)))
            want = oracle.surrogate_uncanon(code[net_pts], y)
            assert np.max(np.abs(got[net_pts] - want)) <= 2e-2 * np.abs(want).max(), b
        n_net += int(net_pts.sum())
    assert n_net > 1000
    batch.close()
    exact.close()
