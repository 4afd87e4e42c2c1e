"""Dense-array twin of the sparse oracle, for brute-force pins on tiny grids.

The sparse oracle reaches neighbours through the package table and the index
shift of Listing 2.  Here the same field is scattered into one dense fine
array (active packages copied, far cells filled with -F / +F by their sign,
a +F border standing for everything outside the domain) and every stencil is
plain array slicing.  With the same sequence of IEEE operations per point the
two must agree bit for bit; any mistake in the tables or the index shift shows
up as a mismatch.  Independent of the oracle's code: numpy only.
"""
import numpy as np

PAD = 4


def to_dense(spec, cell_pkg, cell_type, field, far, far_in=None):
    """Dense copy of a package field; far cells get -far (inside) / +far
    (outside and the border), or far_in / far when far_in is given."""
    nx, ny, nz = spec.dims
    lo_v = -far if far_in is None else far_in
    D = np.full((4 * nz + 2 * PAD, 4 * ny + 2 * PAD, 4 * nx + 2 * PAD), far, dtype=np.float64)
    ct = np.asarray(cell_type).reshape(nz, ny, nx)
    cp = np.asarray(cell_pkg).reshape(nz, ny, nx)
    f = np.asarray(field, dtype=np.float64)
    for K in range(nz):
        for J in range(ny):
            for I in range(nx):
                blk = D[PAD + 4 * K:PAD + 4 * K + 4, PAD + 4 * J:PAD + 4 * J + 4, PAD + 4 * I:PAD + 4 * I + 4]
                t = ct[K, J, I]
                if t >= 2:
                    blk[...] = f[cp[K, J, I]].reshape(4, 4, 4)
                else:
                    blk[...] = lo_v if t == 0 else far
    return D


def from_dense(spec, cell_pkg, cell_type, D, P):
    """Gather a dense array back into package-major storage (active packages)."""
    nx, ny, nz = spec.dims
    out = np.zeros((P, 64))
    ct = np.asarray(cell_type).reshape(nz, ny, nx)
    cp = np.asarray(cell_pkg).reshape(nz, ny, nx)
    for K in range(nz):
        for J in range(ny):
            for I in range(nx):
                if ct[K, J, I] >= 2:
                    out[cp[K, J, I]] = D[PAD + 4 * K:PAD + 4 * K + 4, PAD + 4 * J:PAD + 4 * J + 4,
                                         PAD + 4 * I:PAD + 4 * I + 4].reshape(64)
    return out


def sh(D, dx, dy, dz):
    """View of D shifted by (dx, dy, dz) over the interior region."""
    Z, Y, X = D.shape
    return D[PAD + dz:Z - PAD + dz, PAD + dy:Y - PAD + dy, PAD + dx:X - PAD + dx]


AXES = ((1, 0, 0), (0, 1, 0), (0, 0, 1))


def gradient(D, h):
    c = sh(D, 0, 0, 0)
    inv2h = 1.0 / (2.0 * h)
    out = []
    for e in AXES:
        pl = sh(D, *e) - c
        mi = c - sh(D, -e[0], -e[1], -e[2])
        out.append((pl + mi) * inv2h)
    return out


def laplacian(D, h):
    c = sh(D, 0, 0, 0)
    s = np.zeros_like(c)
    for e in AXES:
        s = s + ((sh(D, *e) - 2.0 * c) + sh(D, -e[0], -e[1], -e[2]))
    return s * (1.0 / (h * h))


def reinit_step(D, D0, S0, h, dt):
    c = sh(D, 0, 0, 0)
    p0 = sh(D0, 0, 0, 0)
    s0 = sh(S0, 0, 0, 0)
    inv_h = 1.0 / h
    G = np.zeros_like(c)
    for e in AXES:
        a = (c - sh(D, -e[0], -e[1], -e[2])) * inv_h
        b = (sh(D, *e) - c) * inv_h
        u = np.where(p0 > 0.0, np.maximum(a, 0.0), np.minimum(a, 0.0))
        v = np.where(p0 > 0.0, np.minimum(b, 0.0), np.maximum(b, 0.0))
        G = G + np.where(u * u > v * v, u * u, v * v)
    return np.where(p0 == 0.0, c, c - dt * s0 * (np.sqrt(G) - 1.0))


def heaviside(z, eps):
    mid = 0.5 * (1.0 + z / eps + np.sin(np.pi * z / eps) / np.pi)
    return np.where(z < -eps, 0.0, np.where(z > eps, 1.0, mid))


def kernel_integrals(D, h):
    """5^3 offsets with the Wendland C2 kernel of support 2h (zero beyond)."""
    num = 0.0
    den = 0.0
    g = [0.0, 0.0, 0.0]
    for sz in range(-2, 3):
        for sy in range(-2, 3):
            for sx in range(-2, 3):
                q = np.sqrt(float(sx * sx + sy * sy + sz * sz))
                if q >= 2.0:
                    continue
                t = 1.0 - 0.5 * q
                w = t ** 4 * (1.0 + 2.0 * q)
                H = heaviside(-sh(D, sx, sy, sz), h)
                num = num + w * H
                den = den + w
                if q > 0:
                    dw = -5.0 * q * t ** 3 / q
                    g[0] = g[0] + dw * (-sx) * H
                    g[1] = g[1] + dw * (-sy) * H
                    g[2] = g[2] + dw * (-sz) * H
    return num / den, g[0] / den, g[1] / den, g[2] / den
