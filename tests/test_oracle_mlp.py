"""Pins of the oracle's surrogate network (FP64) and its inputs."""
import math

import numpy as np
import pytest

import oracle
import sg_inputs as si


def _rand(seed, n):
    st = si.Stream(seed)
    x = 2.0 * st.uniform53(n * 27).reshape(n, 27) - 1.0
    t = st.uniform53(n * 4).reshape(n, 4) - 0.5
    return x, t


def test_gradient_matches_central_differences():
    par = si.mlp_init_params(7).astype(np.float64)
    x, t = _rand(3, 17)
    loss, g = oracle.mlp_loss_grad(par, x, t)
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.choice(np.arange(0, 1728), 40), rng.choice(np.arange(1728, 6212), 60),
                          np.arange(6208, 6212)])
    for k in idx:
        e = 1e-6 * max(1.0, abs(par[k]))
        pp, pm = par.copy(), par.copy()
        pp[k] += e
        pm[k] -= e
        fd = (oracle.mlp_loss_grad(pp, x, t)[0] - oracle.mlp_loss_grad(pm, x, t)[0]) / (2 * e)
        assert abs(fd - g[k]) <= 1e-6 * max(abs(g[k]), 1e-3), (k, fd, g[k])


def test_forward_closed_form_single_path():
    """One active path input 0 -> unit 0 -> unit 0 -> output 0: y0 = silu(silu(x0))."""
    par = np.zeros(oracle.mlp_nparam())
    W1, b1, W2, b2, W3, b3 = oracle.mlp_unpack(par)
    W1[0, 0] = 1.0
    W2[0, 0] = 1.0
    W3[0, 0] = 1.0
    b3[:] = [0.5, -0.25, 0.0, 0.125]
    silu = lambda z: z / (1.0 + math.exp(-z))  # noqa: E731
    x = np.zeros((3, 27))
    x[:, 0] = [0.0, 1.0, -0.7]
    y = oracle.mlp_forward(par, x)
    for r in range(3):
        assert abs(y[r, 0] - (0.5 + silu(silu(x[r, 0])))) < 1e-15
        assert list(y[r, 1:]) == [-0.25, 0.0, 0.125]
    assert abs(silu(1.0) - 0.7310585786300049) < 1e-15


def test_zero_network_outputs_bias_and_bias_gradient():
    par = np.zeros(oracle.mlp_nparam())
    par[-4:] = [0.1, 0.2, 0.3, 0.4]
    x, t = _rand(5, 10)
    y = oracle.mlp_forward(par, x)
    assert np.all(y == par[-4:])
    loss, g = oracle.mlp_loss_grad(par, x, t)
    # dL/db3 = 2 mean over rows (y - t) / 4
    assert np.allclose(g[-4:], 2.0 * (par[-4:] - t).mean(axis=0) / 4.0, atol=1e-15)
    assert abs(loss - ((par[-4:] - t) ** 2).mean()) < 1e-15


def test_adam_first_step_closed_form():
    """Step 1: bias-corrected moments are g and g^2, the update is lr g/(|g| + eps)."""
    par = np.array([0.5, -1.0, 2.0])
    g = np.array([0.3, -2e-3, 0.0])
    m, v = np.zeros(3), np.zeros(3)
    oracle.adam_step(par, g, m, v, lr=1e-2, step=1)
    expect = np.array([0.5, -1.0, 2.0]) - 1e-2 * g / (np.abs(g) + 1e-8)
    assert np.allclose(par, expect, atol=1e-15)


def test_surrogate_inputs_are_clipped_neighbours():
    shape, spec = si.sphere_small()
    G = oracle.build_grid(spec, shape)
    x = oracle.surrogate_inputs(spec, G.nbr, G.phi)
    assert np.all(np.abs(x[2:]) <= 1.0)
    # the centre input (n = 13) is phi / h clipped
    assert np.allclose(x[2:, :, 13], np.clip(G.phi[2:] / spec.h, -1, 1), atol=0)


def test_integrals_are_a_function_of_the_clipped_inputs():
    """The exact integral only sees phi through clip(phi / h): W is the
    class-weighted sum of H(-v) with H(z) = (1 + z + sin(pi z)/pi) / 2."""
    shape, spec = si.sphere_small()
    G = oracle.build_grid(spec, shape)
    x = oracle.surrogate_inputs(spec, G.nbr, G.phi)[2:].reshape(-1, 27)
    W = oracle.kernel_integrals(spec, G.nbr, G.phi)[0][2:].reshape(-1)
    q2 = np.array([(n % 3 - 1) ** 2 + ((n // 3) % 3 - 1) ** 2 + (n // 9 - 1) ** 2 for n in range(27)])
    w = np.array([oracle.wendland(math.sqrt(q)) for q in q2])
    H = 0.5 * (1.0 - x - np.sin(np.pi * x) / np.pi)
    assert np.max(np.abs(H @ w / w.sum() - W)) < 1e-14


def _all_active_grid():
    """A dyadic grid (h = 1/32) on which every background cell is active, so
    that every tap of every interior data point is a data point."""
    spec = si.GridSpec((-0.375, -0.375, -0.375), (6, 6, 6), 1.0 / 32)
    G = oracle.build_grid(spec, si.sphere(0.25, (0.0, 0.0, 0.0)))
    assert G.P == 2 + 6 ** 3
    nx = spec.dims[0]
    pc = G.pkg_cell.astype(np.int64)
    I, J, K = pc % nx, (pc // nx) % nx, pc // (nx * nx)
    d = np.arange(64)
    X = [spec.lo[a] + (4 * c[:, None] + l + 0.5) * spec.h for a, (c, l) in
         enumerate(((I, d % 4), (J, (d // 4) % 4), (K, d // 16)))]
    return spec, G, X


def test_surrogate_class_trivial_at_the_half_width():
    """The Heaviside saturates at |phi| >= h: a field of exactly +h (-h) is
    trivially outside (inside); a field one float below h in magnitude is
    fallback (|phi| < h at the point)."""
    spec, G, _ = _all_active_grid()
    h = np.float32(spec.h)
    assert float(h) == spec.h
    act = slice(2, None)
    for val, want in ((h, 1), (-h, 0), (2 * h, 1), (np.nextafter(h, np.float32(0)), 2),
                      (-np.nextafter(h, np.float32(0)), 2)):
        phi = np.full((G.P, 64), val, np.float32)
        cls = oracle.surrogate_class(spec, G.nbr, phi)
        assert np.all(cls[act] == want), (val, want)
        assert np.all(cls[:2] == 255)


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_surrogate_class_curvature_bound(sign):
    """phi = s (1.5 h + 0.7 (x - x0) + kappa |x - x0|^2 / 6): the 7-point
    Laplacian of a quadratic is exact, kappa; the centre value 1.5 h is not
    fallback by |phi|, the tap at -x (0.8 h + ...) keeps the point
    non-trivial.  |kappa| h just above 0.1 is fallback, just below network."""
    spec, G, X = _all_active_grid()
    h = spec.h
    p0, d0 = 2 + 2 + 6 * (2 + 6 * 2), 1 + 4 * 2 + 16 * 1  # a data point deep inside the all-active grid
    x0 = [X[a][p0, d0] for a in range(3)]
    r2 = sum((X[a] - x0[a]) ** 2 for a in range(3))
    for kh, want in ((0.1 * (1 + 1e-3), 2), (0.1 * (1 - 1e-3), 3), (-0.1 * (1 + 1e-3), 2),
                     (-0.1 * (1 - 1e-3), 3), (0.0, 3)):
        kap = kh / h
        phi = (sign * (1.5 * h + 0.7 * (X[0] - x0[0]) + kap * r2 / 6.0)).astype(np.float32)
        cls, ties = oracle.surrogate_class(spec, G.nbr, phi, ties=True)
        assert cls[p0, d0] == want, (kh, sign, cls[p0, d0])
        assert ties == 0


def _integrals_of_inputs(x):
    """(W, G^) of rows of 27 clipped inputs v by the definitions: W = sum of
    w_s H(-v_s) over the sum of w_s, G^ = sum of w'(|s|) (-s/|s|) H(-v_s)
    over the same sum, H(z) = (1 + z + sin(pi z)/pi) / 2."""
    s = np.array([(n % 3 - 1, (n // 3) % 3 - 1, n // 9 - 1) for n in range(27)], np.float64)
    q = np.sqrt((s ** 2).sum(1))
    w = np.array([oracle.wendland(v) for v in q])
    dw = np.array([oracle.wendland_dq(v) / v if v > 0 else 0.0 for v in q])
    H = 0.5 * (1.0 - x - np.sin(np.pi * x) / np.pi)
    W = H @ w / w.sum()
    G = H @ (dw[:, None] * -s) / w.sum()
    return np.concatenate([W[:, None], G], 1)


@pytest.mark.parametrize("case", ["sphere", "torus_rot"])
def test_surrogate_canonical_frame_is_a_symmetry(case):
    """The integrals of the canonical inputs, carried back by the frame,
    equal the integrals of the point (so the sign, reflection and
    permutation of every frame are a symmetry of W and G^); the canonical
    centre value is >= 0 and the canonical central differences are >= 0."""
    if case == "sphere":
        shape, spec = si.sphere_small()
    else:
        shape = si.torus(0.45, 0.15, rot=si.random_rotation(si.Stream(21)))
        spec = si.GridSpec((-0.8,) * 3, (20, 20, 20), 0.02)
    G = oracle.build_grid(spec, shape)
    phi32 = G.phi.astype(np.float32)
    x, code = oracle.surrogate_canonical(spec, G.nbr, phi32)
    ref = np.stack(oracle.kernel_integrals(spec, G.nbr, phi32.astype(np.float64)), -1)[2:].reshape(-1, 4)
    xc = x[2:].reshape(-1, 27)
    got = oracle.surrogate_uncanon(code[2:].reshape(-1), _integrals_of_inputs(xc))
    assert np.max(np.abs(got - ref)) < 1e-13
    assert np.all(xc[:, 13] >= 0)
    for a, (plus, minus) in enumerate(((14, 12), (16, 10), (22, 4))):
        assert np.all(xc[:, plus] - xc[:, minus] >= 0), a
    # every one of the 48 frames occurs on these bodies except where symmetry forbids; many do
    assert len(np.unique(code[2:] >> 1)) >= 24
