"""Pins of the grid options of the oracle: kernel support, Heaviside half
width and package id order.

* Wendland C2 of support R = 3 against values worked out by hand from its
  definition (1 - q/R)^4 (1 + 4q/R): w(0) = 1, w(1) = 112/243, w(2) = 11/243,
  w'(1) = -160/243, zero at q >= 3.
* For any support and half width: W = 1/2 at a plane through a data layer
  (H(-z) = 1 - H(z) and the taps pair up; to rounding, the numerator and the
  denominator sum the taps in different orders), 1 and 0 exactly deep inside
  and far outside (there the two sums are the same sum), G = 0 to rounding.
* Package ids in Morton order: a relabelling only; gradient, reinit and
  integrals of every cell are the same as with linear ids, bit for bit.
"""
import numpy as np
import pytest

import oracle
import sg_inputs as si


def test_wendland_support3_closed_form():
    assert oracle.wendland_r(0.0, 3.0) == 1.0
    assert oracle.wendland_r(1.0, 3.0) == pytest.approx(112.0 / 243.0, rel=1e-15)
    assert oracle.wendland_r(2.0, 3.0) == pytest.approx(11.0 / 243.0, rel=1e-15)
    assert oracle.wendland_r_dq(1.0, 3.0) == pytest.approx(-160.0 / 243.0, rel=1e-15)
    assert oracle.wendland_r(3.0, 3.0) == 0.0 and oracle.wendland_r(3.2, 3.0) == 0.0
    # support 2 reduces to the default kernel
    for q in (0.0, 0.5, 1.0, 1.4142135623730951, 1.7320508075688772, 2.0):
        assert oracle.wendland_r(q, 2.0) == pytest.approx(oracle.wendland(q), rel=1e-15, abs=1e-300)
        assert oracle.wendland_r_dq(q, 2.0) == pytest.approx(oracle.wendland_dq(q), rel=1e-15, abs=1e-300)


@pytest.mark.parametrize("R,e", [(1.5, 1.0), (2.5, 1.0), (3.0, 2.0), (2.0, 0.5)])
def test_plane_half_and_deep_values(R, e):
    h = 2.0 ** -5
    shape = si.plane((0.0, 0.0, 1.0), point=(0.0, 0.0, 0.5 * h))  # through a data layer
    spec = si.GridSpec((-0.5, -0.5, -0.5), (8, 8, 8), h, kernel_support=R * h, heaviside_eps=e * h)
    G = oracle.build_grid(spec, shape)
    Wf = oracle.kernel_integrals(spec, G.nbr, G.phi)
    interior = (G.pkg_type >= 2) & np.all(G.nbr >= 2, axis=1)
    d = np.abs(G.phi)
    on = interior[:, None] & (d < 1e-12)
    assert on.sum() > 50
    assert np.max(np.abs(Wf[0][on] - 0.5)) <= 1e-15
    assert np.max(np.abs(Wf[1][on])) < 1e-15 and np.max(np.abs(Wf[2][on])) < 1e-15
    # every tap (|s_z| <= 2) of these points saturates H, far packages included;
    # taps leaving the domain sideways would read the outside package
    nx, ny, _ = spec.dims
    pc = np.maximum(G.pkg_cell, 0).astype(np.int64)
    dd = np.arange(64)
    xi = 4 * (pc % nx)[:, None] + (dd % 4)[None, :]
    yi = 4 * ((pc // nx) % ny)[:, None] + ((dd // 4) % 4)[None, :]
    lateral = (xi >= 2) & (xi <= 4 * nx - 3) & (yi >= 2) & (yi <= 4 * ny - 3)
    deep = (np.arange(G.P) >= 2)[:, None] & lateral & (d > (2 + e) * h + 1e-12)
    inside = deep & (G.phi < 0)
    outside = deep & (G.phi > 0)
    assert inside.sum() > 20 and outside.sum() > 20
    assert np.all(Wf[0][inside] == 1.0) and np.all(Wf[0][outside] == 0.0)
    for a in (1, 2, 3):  # the signed taps cancel to rounding
        assert np.max(np.abs(Wf[a][deep])) <= 1e-15


def test_morton_ids_are_a_relabelling():
    shape = si.torus(0.5, 0.18, rot=si.random_rotation(si.Stream(3)))
    spec0 = si.GridSpec((-0.8, -0.8, -0.8), (16, 16, 16), 0.025)
    spec1 = si.GridSpec(spec0.lo, spec0.dims, spec0.h, id_order=1)
    A, B = oracle.build_grid(spec0, shape), oracle.build_grid(spec1, shape)
    assert A.P == B.P
    act = A.cell_pkg >= 2
    assert np.array_equal(act, B.cell_pkg >= 2)
    assert np.array_equal(A.cell_pkg[~act], B.cell_pkg[~act])
    assert np.array_equal(np.sort(B.cell_pkg[act]), np.arange(2, A.P))
    # ids increase along the Morton order of the cells
    nx, ny, _ = spec0.dims
    c = np.nonzero(act)[0]
    I, J, K = c % nx, (c // nx) % ny, c // (nx * ny)
    key = np.zeros(c.size, np.int64)
    for b in range(5):
        key |= ((I >> b) & 1) << (3 * b) | ((J >> b) & 1) << (3 * b + 1) | ((K >> b) & 1) << (3 * b + 2)
    assert np.all(np.diff(B.cell_pkg[c][np.argsort(key)]) == 1)
    # the per-cell fields do not depend on the labelling
    perm = np.empty(A.P, np.int64)
    perm[:2] = [0, 1]
    perm[A.cell_pkg[act]] = B.cell_pkg[act]  # package of A -> package of B
    for fa, fb in ((A.phi, B.phi), (oracle.gradient(spec0, A.nbr, A.phi)[1], oracle.gradient(spec1, B.nbr, B.phi)[1]),
                   (oracle.reinit(spec0, A.nbr, A.phi, 5, 0.5), oracle.reinit(spec1, B.nbr, B.phi, 5, 0.5)),
                   (oracle.kernel_integrals(spec0, A.nbr, A.phi)[0], oracle.kernel_integrals(spec1, B.nbr, B.phi)[0])):
        assert np.array_equal(fa, fb[perm])


@pytest.mark.parametrize("R,e", [(3.0, 2.0), (1.5, 1.0), (2.5, 0.5)])
def test_plane_reduces_to_column_sums(R, e):
    """At a plane z = c the tap sum depends on s_z only: W = sum_sz C(sz) H(-(d + sz h)) / sum C,
    G_z = sum_sz D(sz) (-sz) H / sum C with the column sums C(sz) = sum_{sx,sy} w(q) and
    D(sz) = sum_{sx,sy} w'(q)/q (closed-form kernel pinned above)."""
    h = 2.0 ** -5
    for frac in (0.25, 0.5, 0.875):
        shape = si.plane((0.0, 0.0, 1.0), point=(0.0, 0.0, frac * h))
        spec = si.GridSpec((-0.5, -0.5, -0.5), (8, 8, 8), h, kernel_support=R * h, heaviside_eps=e * h)
        G = oracle.build_grid(spec, shape)
        Wf = oracle.kernel_integrals(spec, G.nbr, G.phi)
        Cs, Ds = {}, {}
        for sz in range(-2, 3):
            c = dsum = 0.0
            for sx in range(-2, 3):
                for sy in range(-2, 3):
                    q = (sx * sx + sy * sy + sz * sz) ** 0.5
                    c += oracle.wendland_r(q, R)
                    if q > 0:
                        dsum += oracle.wendland_r_dq(q, R) / q
            Cs[sz], Ds[sz] = c, dsum
        den = sum(Cs.values())
        interior = (G.pkg_type >= 2) & np.all(G.nbr >= 2, axis=1)
        checked = 0
        for p in np.nonzero(interior)[0][:40]:
            for dd in range(64):
                d = G.phi[p, dd]  # signed distance of the data point
                H = {sz: oracle.heaviside(-(d + sz * h), e * h) for sz in range(-2, 3)}
                Wr = sum(Cs[sz] * H[sz] for sz in H) / den
                Gr = sum(Ds[sz] * (-sz) * H[sz] for sz in H) / den
                assert abs(Wf[0][p, dd] - Wr) < 1e-14
                assert abs(Wf[3][p, dd] - Gr) < 1e-14
                checked += 1
        assert checked > 1000
