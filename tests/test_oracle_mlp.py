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
