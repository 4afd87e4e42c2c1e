"""The surrogate network and the surrogate kernel integrals on the GPU.

Forward and gradients against the FP64 oracle on the same BF16-rounded
weights and inputs; classification against the oracle's FP64 decision;
trivial and fallback points against the exact integrals; network points
against the oracle network on the oracle's canonical inputs; sample
gathering in the canonical frame; reproducible training.
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


def bf16_round(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def rows32(x27):
    x = np.zeros((x27.shape[0], 32), np.float32)
    x[:, :27] = x27
    return torch.from_numpy(x).to(torch.bfloat16).cuda()


def _data(seed, n):
    st = si.Stream(seed)
    x = 2.0 * st.uniform53(n * 27).reshape(n, 27) - 1.0
    t = st.uniform53(n * 4).reshape(n, 4) - 0.5
    return x, t


def test_forward_matches_oracle(sg):
    par = si.mlp_init_params(11)
    net = sg.MLP(par)
    x, _ = _data(1, 1003)
    X = rows32(x)
    y = net.forward(X).cpu().numpy().astype(np.float64)
    ref = oracle.mlp_forward(bf16_round(par), X.float().cpu().numpy()[:, :27].astype(np.float64))
    scale = np.abs(ref).max()
    assert np.max(np.abs(y - ref)) <= 2e-2 * scale
    assert np.sqrt(np.mean((y - ref) ** 2)) <= 5e-3 * scale
    assert np.allclose(net.get_params(), par)


@pytest.mark.parametrize("n", [64, 200, 8192])
def test_gradient_matches_oracle(sg, n):
    par = si.mlp_init_params(12)
    net = sg.MLP(par)
    x, t = _data(2, n)
    X = rows32(x)
    T = torch.from_numpy(t.astype(np.float32)).cuda()
    g, loss = net.loss_grad(X, T)
    g = g.cpu().numpy().astype(np.float64)
    xr = X.float().cpu().numpy()[:, :27].astype(np.float64)
    lref, gref = oracle.mlp_loss_grad(bf16_round(par), xr, t.astype(np.float32).astype(np.float64))
    assert abs(loss.item() - lref) <= 2e-2 * lref
    assert np.linalg.norm(g - gref) <= 2e-2 * np.linalg.norm(gref)
    # per block: every layer's gradient, not only the large ones
    for a, b in ((0, 1728), (1728, 1792), (1792, 5888), (5888, 5952), (5952, 6208), (6208, 6212)):
        assert np.linalg.norm(g[a:b] - gref[a:b]) <= 2e-2 * np.linalg.norm(gref[a:b]) + 1e-9


def test_gradient_with_index_rows(sg):
    par = si.mlp_init_params(13)
    net = sg.MLP(par)
    x, t = _data(3, 500)
    X = rows32(x)
    T = torch.from_numpy(t.astype(np.float32)).cuda()
    idx = torch.from_numpy(np.random.default_rng(1).permutation(500)[:300].astype(np.int32)).cuda()
    g1, _ = net.loss_grad(X, T, idx)
    g2, _ = net.loss_grad(X[idx.long()].contiguous(), T[idx.long()].contiguous())
    assert torch.allclose(g1, g2, rtol=1e-4, atol=1e-9)


def test_train_step_matches_oracle_adam(sg):
    par = si.mlp_init_params(14)
    net = sg.MLP(par)
    x, t = _data(4, 256)
    X = rows32(x)
    T = torch.from_numpy(t.astype(np.float32)).cuda()
    g, _ = net.loss_grad(X, T)
    net.train_step(X, T, None, 1e-3)
    got = net.get_params().astype(np.float64)
    p = par.astype(np.float64)
    m, v = np.zeros_like(p), np.zeros_like(p)
    oracle.adam_step(p, g.cpu().numpy().astype(np.float64), m, v, lr=1e-3, step=1)
    assert np.max(np.abs(got - p)) <= 1e-6


def test_many_ctas_gradient_and_adam(sg):
    """70,000 rows are 547 CTAs of 128: the partial gradients are summed in
    several blocks of 128 CTAs and a ragged rest.  Against the oracle; every
    row twice gives the same mean loss and gradient (a block of partials
    dropped or counted twice would not); the Adam kernel's own sum of the
    partials gives the oracle's Adam step from the summed gradient."""
    n = 70_000
    par = si.mlp_init_params(15)
    net = sg.MLP(par)
    x, t = _data(8, n)
    X = rows32(x)
    T = torch.from_numpy(t.astype(np.float32)).cuda()
    g, loss = net.loss_grad(X, T)
    gd = g.cpu().numpy().astype(np.float64)
    xr = X.float().cpu().numpy()[:, :27].astype(np.float64)
    lref, gref = oracle.mlp_loss_grad(bf16_round(par), xr, t.astype(np.float32).astype(np.float64))
    assert abs(loss.item() - lref) <= 2e-2 * lref
    assert np.linalg.norm(gd - gref) <= 2e-2 * np.linalg.norm(gref)
    g2, loss2 = net.loss_grad(torch.cat([X, X]), torch.cat([T, T]))
    assert abs(loss2.item() - loss.item()) <= 1e-5 * loss.item()
    assert np.linalg.norm(g2.cpu().numpy().astype(np.float64) - gd) <= 1e-5 * np.linalg.norm(gd)
    net.train_step(X, T, None, 1e-3)
    got = net.get_params().astype(np.float64)
    p = par.astype(np.float64)
    m, v = np.zeros_like(p), np.zeros_like(p)
    oracle.adam_step(p, gd, m, v, lr=1e-3, step=1)
    assert np.max(np.abs(got - p)) <= 1e-6


def test_training_is_reproducible(sg):
    """The partial gradients of the CTAs are summed in a fixed order: two
    trainings from the same start on the same batches end bit for bit equal."""
    x, t = _data(6, 4096)
    X = rows32(x)
    T = torch.from_numpy(t.astype(np.float32)).cuda()
    idx = torch.from_numpy(np.random.default_rng(2).permutation(4096)[:2500].astype(np.int32)).cuda()
    out = []
    for _ in range(2):
        net = sg.MLP(si.mlp_init_params(17))
        for s in range(20):
            net.train_step(X, T, idx if s % 2 else None, 2e-3)
        out.append(net.get_params())
    assert np.array_equal(out[0], out[1])


def test_training_reduces_loss(sg):
    net = sg.MLP(si.mlp_init_params(15))
    x, t = _data(5, 8192)
    # a smooth target: the exact integral's structure (sum of a 1-D function of the inputs)
    H = 0.5 * (1.0 - x - np.sin(np.pi * x) / np.pi)
    t = np.stack([H.mean(1), H[:, 14] - H[:, 12], H[:, 16] - H[:, 10], H[:, 22] - H[:, 4]], 1)
    X = rows32(x)
    T = torch.from_numpy(t.astype(np.float32)).cuda()
    _, l0 = net.loss_grad(X, T)
    for _ in range(300):
        net.train_step(X, T, None, 3e-3)
    _, l1 = net.loss_grad(X, T)
    assert l1.item() < 0.05 * l0.item()


def _grid(sg, shape, spec, iters=5):
    g = sg.Grid(spec)
    g.tag_allocate(shape)
    g.init_sdf(shape)
    g.reinit(iters, 0.5)
    return g


CASES = {
    "sphere_small": si.sphere_small(),
    "torus_rot": (si.torus(0.45, 0.15, rot=si.random_rotation(si.Stream(21))), si.GridSpec((-0.8,) * 3, (20, 20, 20), 0.02)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_classification_matches_oracle(sg, name):
    shape, spec = CASES[name]
    g = _grid(sg, shape, spec)
    cls = g.surrogate_classify().cpu().numpy()
    phi = g.field("phi").cpu().numpy()
    ref, ties = oracle.surrogate_class(spec, g.field("nbr").cpu().numpy(), phi, ties=True)
    assert ties == 0
    assert np.array_equal(cls, ref)
    assert set(np.unique(cls[2:])) <= {0, 1, 2, 3} and (cls[2:] == 3).sum() > 0


@pytest.mark.parametrize("name", list(CASES))
def test_surrogate_integrals(sg, name):
    shape, spec = CASES[name]
    g = _grid(sg, shape, spec)
    g.kernel_integrals()
    exact = {f: g.field(f).clone() for f in ("W", "Gx", "Gy", "Gz")}
    par = si.mlp_init_params(16)
    net = sg.MLP(par)
    g.kernel_integrals(mode=1, mlp=net)
    cls = g.surrogate_classify()
    stats = g.surrogate_stats()
    counts = [int((cls[2:] == c).sum()) for c in range(4)]
    assert stats == counts
    fb = cls == 2
    for f in ("W", "Gx", "Gy", "Gz"):
        got = g.field(f)
        assert torch.equal(got[fb], exact[f][fb])  # fallback: the exact sum, bit for bit
    tin, tout = cls == 0, cls == 1
    assert torch.all(g.field("W")[tin] == 1) and torch.all(g.field("W")[tout] == 0)
    for f in ("Gx", "Gy", "Gz"):
        assert torch.all(g.field(f)[tin | tout] == 0)
    # network points against the oracle network on the oracle's canonical inputs, carried back
    phi = g.field("phi").cpu().numpy()
    xin, code = oracle.surrogate_canonical(spec, g.field("nbr").cpu().numpy(), phi)
    net_pts = (cls == 3).cpu().numpy()
    xr = bf16_round(xin[net_pts].astype(np.float32))
    ref = oracle.surrogate_uncanon(code[net_pts], oracle.mlp_forward(bf16_round(par), xr))
    got = np.stack([g.field(f).cpu().numpy()[net_pts] for f in ("W", "Gx", "Gy", "Gz")], 1)
    scale = np.abs(ref).max()
    assert np.max(np.abs(got - ref)) <= 2e-2 * scale


def test_surrogate_samples(sg):
    """Samples are the network points in point order: canonical inputs (the
    oracle's frame, BF16) and the exact integrals carried into that frame."""
    shape, spec = CASES["torus_rot"]
    g = _grid(sg, shape, spec)
    g.kernel_integrals()
    x, t, n = g.surrogate_samples(seed=4, keep=1.0)
    cls = g.surrogate_classify().cpu().numpy()
    sel = cls == 3
    assert n == sel.sum() == x.shape[0]
    xin, code = oracle.surrogate_canonical(spec, g.field("nbr").cpu().numpy(), g.field("phi").cpu().numpy())
    xin, code = xin[sel], code[sel]
    assert np.max(np.abs(x.float().cpu().numpy()[:, :27] - bf16_round(xin.astype(np.float32)))) <= 1e-6
    assert torch.all(x[:, 27:] == 0)
    exact = np.stack([g.field(f).cpu().numpy()[sel] for f in ("W", "Gx", "Gy", "Gz")], 1).astype(np.float64)
    back = oracle.surrogate_uncanon(code, t.cpu().numpy())
    assert np.max(np.abs(back - exact)) <= 1e-7
    # the frame permutes and negates the components of G^: their magnitudes are kept exactly
    assert np.array_equal(np.sort(np.abs(t[:, 1:].cpu().numpy()), 1), np.sort(np.abs(exact[:, 1:]), 1).astype(np.float32))
    # sub-sampling keeps a deterministic subset of about the requested size
    x2, t2, n2 = g.surrogate_samples(seed=4, keep=0.25)
    x3, t3, n3 = g.surrogate_samples(seed=4, keep=0.25)
    assert n2 == n3 and torch.equal(x2, x3)
    assert 0.15 * n < n2 < 0.35 * n
    x4, _, n4 = g.surrogate_samples(seed=4, keep=1.0, cap=100)
    assert n4 == n and x4.shape[0] == 100 and torch.equal(x4, x[:100])
