"""FP64 CPU oracle of the sparse narrow-band level-set grid (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU baseline use this
package.  It wraps ``sg_oracle.c`` (plain loops in double precision, see the
header of that file for the passages each routine follows) through ctypes and
shares no code with the CUDA library.  Arrays are numpy, package-major with
64 values per package (in-package index d = i + 4j + 16k).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import types

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

SPHERE, PLANE, TORUS, PRISM, ROUNDED_BOX, SHELL = 0, 1, 2, 3, 4, 5


def build(force: bool = False) -> str:
    """Compile sg_oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                               "-std=c11", "-D_DEFAULT_SOURCE", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Shape(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad", C.c_int32), ("centre", C.c_double * 3),
                ("rot", C.c_double * 9), ("p", C.c_double * 8)]


class _Grid(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("dims", C.c_int32 * 3), ("id_order", C.c_int32),
                ("h", C.c_double), ("far_value", C.c_double), ("support", C.c_double), ("eps", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.or_tag.restype = C.c_int64
        _lib.or_tag_from.restype = C.c_int64
        _lib.or_sdf.restype = C.c_double
        _lib.or_sdf.argtypes = [C.POINTER(_Shape), C.c_double, C.c_double, C.c_double]
        _lib.or_get_threads.restype = C.c_int
        for f in ("or_wendland_r", "or_wendland_r_dq"):
            getattr(_lib, f).restype = C.c_double
            getattr(_lib, f).argtypes = [C.c_double, C.c_double]
        for f in ("or_wendland", "or_wendland_dq"):
            getattr(_lib, f).restype = C.c_double
            getattr(_lib, f).argtypes = [C.c_double]
        _lib.or_lattice_ties.restype = C.c_int64
        _lib.or_heaviside.restype = C.c_double
        _lib.or_heaviside.argtypes = [C.c_double, C.c_double]
    return _lib


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def get_threads() -> int:
    return int(lib().or_get_threads())


def _shape(s) -> _Shape:
    out = _Shape()
    out.kind = int(s.kind)
    out.centre[:] = list(s.centre)
    out.rot[:] = list(s.rot)
    out.p[:] = list(s.p)
    return out


def far_value(spec) -> float:
    """F = 4 lc = 16 h: larger than any active |phi| of the +-2 cell band."""
    return 16.0 * float(spec.h)


def _grid(spec, far=None) -> _Grid:
    g = _Grid()
    g.lo[:] = [float(v) for v in spec.lo]
    g.dims[:] = [int(v) for v in spec.dims]
    g.h = float(spec.h)
    g.far_value = far_value(spec) if far is None else float(far)
    g.support = float(getattr(spec, "kernel_support", 0.0) or 0.0)
    g.eps = float(getattr(spec, "heaviside_eps", 0.0) or 0.0)
    g.id_order = int(getattr(spec, "id_order", 0) or 0)
    return g


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def sdf(shape, x, y, z):
    x, y, z = _f64(x), _f64(y), _f64(z)
    out = np.empty_like(x)
    lib().or_sdf_many(C.byref(_shape(shape)), C.c_int64(x.size), _p(x), _p(y), _p(z), _p(out))
    return out


def wendland(q):
    return lib().or_wendland(float(q))


def wendland_dq(q):
    return lib().or_wendland_dq(float(q))


def wendland_r(q, R):
    """Wendland C2 of support R (units of h)."""
    return lib().or_wendland_r(float(q), float(R))


def wendland_r_dq(q, R):
    return lib().or_wendland_r_dq(float(q), float(R))


def heaviside(z, eps):
    return lib().or_heaviside(float(z), float(eps))


def tag(spec, shape):
    """Returns (cell_pkg int32[nc], cell_type uint8[nc], P, near_ties)."""
    nc = spec.n_cells
    cell_pkg = np.empty(nc, np.int32)
    cell_type = np.empty(nc, np.uint8)
    ties = C.c_int64(0)
    P = lib().or_tag(C.byref(_grid(spec)), C.byref(_shape(shape)), _p(cell_pkg), _p(cell_type), C.byref(ties))
    return cell_pkg, cell_type, int(P), int(ties.value)


def tag_from(spec, shape, coarse_spec, c_cell_pkg, c_pkg_type, c_phi):
    """Tagging of a layer from its coarser layer (same lo, half the dims, twice
    the spacing).  Returns (cell_pkg, cell_type, P, near_ties, evaluated)."""
    nc = spec.n_cells
    cell_pkg = np.empty(nc, np.int32)
    cell_type = np.empty(nc, np.uint8)
    ties, ev = C.c_int64(0), C.c_int64(0)
    P = lib().or_tag_from(C.byref(_grid(spec)), C.byref(_shape(shape)), C.byref(_grid(coarse_spec)),
                          _p(np.ascontiguousarray(c_cell_pkg, np.int32)), _p(np.ascontiguousarray(c_pkg_type, np.uint8)),
                          _p(_f64(c_phi)), _p(cell_pkg), _p(cell_type), C.byref(ties), C.byref(ev))
    return cell_pkg, cell_type, int(P), int(ties.value), int(ev.value)


def tables(spec, cell_pkg, cell_type, P):
    """Returns (pkg_cell int32[P], pkg_type uint8[P], nbr int32[P,27])."""
    pkg_cell = np.empty(P, np.int32)
    pkg_type = np.empty(P, np.uint8)
    nbr = np.empty((P, 27), np.int32)
    lib().or_tables(C.byref(_grid(spec)), _p(np.ascontiguousarray(cell_pkg, np.int32)),
                    _p(np.ascontiguousarray(cell_type, np.uint8)), C.c_int64(P), _p(pkg_cell), _p(pkg_type),
                    _p(nbr))
    return pkg_cell, pkg_type, nbr


def init_sdf(spec, shape, P, pkg_cell, far=None):
    phi = np.empty((P, 64), np.float64)
    lib().or_init_sdf(C.byref(_grid(spec, far)), C.byref(_shape(shape)), C.c_int64(P),
                      _p(np.ascontiguousarray(pkg_cell, np.int32)), _p(phi))
    return phi


def gradient(spec, nbr, phi):
    phi = _f64(phi)
    P = phi.shape[0]
    out = [np.empty((P, 64), np.float64) for _ in range(3)]
    lib().or_gradient(C.byref(_grid(spec)), C.c_int64(P), _p(np.ascontiguousarray(nbr, np.int32)), _p(phi),
                      *[_p(o) for o in out])
    return tuple(out)


def sequential(phi32, delta):
    """phi + delta on the active packages, in float32."""
    phi = np.array(phi32, dtype=np.float32, copy=True, order="C")
    lib().or_sequential(C.c_int64(phi.shape[0]), _p(phi), C.c_float(delta))
    return phi


def laplacian(spec, nbr, phi):
    phi = _f64(phi)
    P = phi.shape[0]
    out = np.empty((P, 64), np.float64)
    lib().or_laplacian(C.byref(_grid(spec)), C.c_int64(P), _p(np.ascontiguousarray(nbr, np.int32)), _p(phi),
                       _p(out))
    return out


def reinit_s0(spec, phi0):
    phi0 = _f64(phi0)
    out = np.empty_like(phi0)
    lib().or_reinit_s0(C.byref(_grid(spec)), C.c_int64(phi0.shape[0]), _p(phi0), _p(out))
    return out


def reinit_step(spec, nbr, phi0, s0, phi_in, dt):
    phi0, s0, phi_in = _f64(phi0), _f64(s0), _f64(phi_in)
    out = np.empty_like(phi_in)
    lib().or_reinit_step(C.byref(_grid(spec)), C.c_int64(phi_in.shape[0]), _p(np.ascontiguousarray(nbr, np.int32)),
                         _p(phi0), _p(s0), _p(phi_in), _p(out), C.c_double(dt))
    return out


def reinit(spec, nbr, phi, iterations, cfl):
    phi = np.array(phi, dtype=np.float64, copy=True, order="C")
    lib().or_reinit(C.byref(_grid(spec)), C.c_int64(phi.shape[0]), _p(np.ascontiguousarray(nbr, np.int32)),
                    _p(phi), C.c_int32(iterations), C.c_double(cfl))
    return phi


def kernel_integrals(spec, nbr, phi):
    phi = _f64(phi)
    P = phi.shape[0]
    out = [np.empty((P, 64), np.float64) for _ in range(4)]
    lib().or_kernel_integrals(C.byref(_grid(spec)), C.c_int64(P), _p(np.ascontiguousarray(nbr, np.int32)),
                              _p(phi), *[_p(o) for o in out])
    return tuple(out)


def probe(spec, cell_pkg, nbr, fields, x, y, z):
    """fields: (phi, gx, gy, gz, W, Gx, Gy, Gz); returns (phi, nx, ny, nz, W, Gx, Gy, Gz)."""
    fs = [_f64(f) for f in fields]
    x, y, z = (np.ascontiguousarray(v, np.float32) for v in (x, y, z))
    n = x.size
    outs = [np.empty(n, np.float64) for _ in range(8)]
    farr = (C.c_void_p * 8)(*[f.ctypes.data for f in fs])
    oarr = (C.c_void_p * 8)(*[o.ctypes.data for o in outs])
    lib().or_probe(C.byref(_grid(spec)), _p(np.ascontiguousarray(cell_pkg, np.int32)),
                   _p(np.ascontiguousarray(nbr, np.int32)), farr, C.c_int64(n), _p(x), _p(y), _p(z), oarr)
    return tuple(outs)


def consistency_correct(spec, P, cell_pkg, pkg_cell, pkg_type, nbr, phi, trust=1.0, sweeps=False):
    """Consistency (sign) correction with trusted band |phi| < trust * h
    (trust * h rounded to float32, as the device takes it).  Returns
    (cell_pkg, nbr, phi, (points flipped, far cells moved)), all copies, and
    with sweeps=True also (point sweeps, cell sweeps), each up to and
    including the first sweep that labels nothing."""
    cp = np.array(cell_pkg, np.int32, copy=True)
    nb = np.array(nbr, np.int32, copy=True, order="C")
    ph = np.array(phi, np.float64, copy=True, order="C")
    ch = (C.c_int64 * 4)()
    tau = float(np.float32(float(np.float32(trust)) * spec.h))  # as the library takes it
    lib().or_consistency_correct(C.byref(_grid(spec)), C.c_int64(int(P)), _p(cp),
                                 _p(np.ascontiguousarray(pkg_cell, np.int32)),
                                 _p(np.ascontiguousarray(pkg_type, np.uint8)), _p(nb), _p(ph), C.c_double(tau), ch)
    if sweeps:
        return cp, nb, ph, (int(ch[0]), int(ch[1])), (int(ch[2]), int(ch[3]))
    return cp, nb, ph, (int(ch[0]), int(ch[1]))


def relax(spec, cell_pkg, nbr, fields, x, y, z, steps, step=0.1):
    """Particle relaxation: `steps` times probe, then move by
    -step h clip(phi/h, -1, 1) n with float32 positions.  Returns the final
    (x, y, z) (float32) and the last step's probe (phi, nx, ny, nz, W, Gx, Gy,
    Gz)."""
    fs = [_f64(f) for f in fields]
    x, y, z = (np.array(v, np.float32, copy=True) for v in (x, y, z))
    n = x.size
    outs = [np.zeros(n, np.float64) for _ in range(8)]
    farr = (C.c_void_p * 8)(*[f.ctypes.data for f in fs])
    oarr = (C.c_void_p * 8)(*[o.ctypes.data for o in outs])
    lib().or_relax(C.byref(_grid(spec)), _p(np.ascontiguousarray(cell_pkg, np.int32)),
                   _p(np.ascontiguousarray(nbr, np.int32)), farr, C.c_int64(n), _p(x), _p(y), _p(z),
                   C.c_int32(int(steps)), C.c_double(float(step)), oarr)
    return (x, y, z), tuple(outs)


def morton_keys(spec, x, y, z):
    x, y, z = (np.ascontiguousarray(v, np.float32) for v in (x, y, z))
    keys = np.empty(x.size, np.uint64)
    lib().or_morton_keys(C.byref(_grid(spec)), C.c_int64(x.size), _p(x), _p(y), _p(z), _p(keys))
    return keys


def lattice_ties(spec, x, y, z, tol=1e-9, mask=False):
    """Number of particles with a lattice coordinate u = (x - lo)/h - 1/2
    within tol of an integer on some axis: their cell decision rests on the
    last bits of the arithmetic.  With mask=True also returns a uint8 array,
    bit a set where axis a is tied."""
    x, y, z = (np.ascontiguousarray(v, np.float32) for v in (x, y, z))
    m = np.zeros(x.size, np.uint8) if mask else None
    n = int(lib().or_lattice_ties(C.byref(_grid(spec)), C.c_int64(x.size), _p(x), _p(y), _p(z), C.c_double(tol),
                                  _p(m) if mask else None))
    return (n, m) if mask else n


def morton_keys_accept(spec, x, y, z, keys):
    """Whether the given Morton keys are the oracle's: equal for every
    particle away from lattice planes; a particle within 1e-9 of a plane on
    some axes (two cell decisions are then both correct) may carry the key of
    either side of each such plane, judged by moving that coordinate one
    float step down or up.  Returns (ok, number of tied particles)."""
    x, y, z = (np.ascontiguousarray(v, np.float32) for v in (x, y, z))
    keys = np.asarray(keys).view(np.uint64)
    n_t, m = lattice_ties(spec, x, y, z, mask=True)
    ref = morton_keys(spec, x, y, z)
    free = m == 0
    if not np.array_equal(keys[free], ref[free]):
        return False, n_t
    for q in np.nonzero(~free)[0]:
        cands = set()
        for c in range(8):
            p = [x[q], y[q], z[q]]
            for a in range(3):
                if m[q] >> a & 1:
                    p[a] = np.nextafter(p[a], np.float32(-np.inf if (c >> a) & 1 else np.inf))
            cands.add(int(morton_keys(spec, *(np.array([v], np.float32) for v in p))[0]))
        if int(keys[q]) not in cands:
            return False, n_t
    return True, n_t


def morton_order(keys):
    keys = np.ascontiguousarray(keys, np.uint64)
    order = np.empty(keys.size, np.int64)
    lib().or_morton_order(C.c_int64(keys.size), _p(keys), _p(order))
    return order


MLP_IN, MLP_H, MLP_OUT = 27, 64, 4


def mlp_nparam():
    lib().or_mlp_nparam.restype = C.c_int64
    return int(lib().or_mlp_nparam())


def mlp_unpack(par):
    """Views W1[64,27], b1, W2[64,64], b2, W3[4,64], b3 of a flat parameter vector."""
    par = np.asarray(par)
    o = 0
    out = []
    for shape in ((MLP_H, MLP_IN), (MLP_H,), (MLP_H, MLP_H), (MLP_H,), (MLP_OUT, MLP_H), (MLP_OUT,)):
        n = int(np.prod(shape))
        out.append(par[o:o + n].reshape(shape))
        o += n
    return out


def mlp_forward(par, x):
    par, x = _f64(par), _f64(x)
    n = x.shape[0]
    y = np.empty((n, MLP_OUT))
    lib().or_mlp_forward(_p(par), C.c_int64(n), _p(x), _p(y), None, None)
    return y


def mlp_loss_grad(par, x, t):
    par, x, t = _f64(par), _f64(x), _f64(t)
    g = np.empty_like(par)
    lib().or_mlp_loss_grad.restype = C.c_double
    loss = lib().or_mlp_loss_grad(_p(par), C.c_int64(x.shape[0]), _p(x), _p(t), _p(g))
    return float(loss), g


def adam_step(par, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8):
    """In place on par, m, v (float64 arrays)."""
    lib().or_adam_step(_p(par), _p(_f64(grad)), _p(m), _p(v), C.c_int64(par.size), C.c_double(lr),
                       C.c_double(beta1), C.c_double(beta2), C.c_double(eps), C.c_int64(step))


def surrogate_inputs(spec, nbr, phi):
    phi = _f64(phi)
    P = phi.shape[0]
    x = np.zeros((P, 64, MLP_IN))
    lib().or_surrogate_inputs(C.byref(_grid(spec)), C.c_int64(P), _p(np.ascontiguousarray(nbr, np.int32)), _p(phi),
                              _p(x))
    return x


def surrogate_canonical(spec, nbr, phi32):
    """Canonical inputs (P, 64, 27) and frame codes (P, 64) of every data
    point of the float field phi32 (see or_surrogate_canonical)."""
    phi32 = np.ascontiguousarray(phi32, np.float32)
    P = phi32.shape[0]
    x = np.zeros((P, 64, MLP_IN))
    code = np.zeros((P, 64), np.int32)
    lib().or_surrogate_canonical(C.byref(_grid(spec)), C.c_int64(P), _p(np.ascontiguousarray(nbr, np.int32)),
                                 _p(phi32), _p(x), _p(code))
    return x, code


_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def surrogate_uncanon(code, y):
    """Outputs (W', G'_0, G'_1, G'_2) in the canonical frames `code` -> (W, G^)
    of the points: W = 1 - W' where the frame negated phi; component k of G'
    belongs to original axis p[k], negated where that axis was reversed or
    phi negated."""
    code = np.asarray(code).reshape(-1)
    y = np.asarray(y, np.float64).reshape(-1, 4)
    flip = (code & 1) == 1
    out = np.empty_like(y)
    out[:, 0] = np.where(flip, 1.0 - y[:, 0], y[:, 0])
    for r, c in enumerate(code):
        q = _PERMS[c >> 4]
        for k in range(3):
            a = q[k]
            neg = bool((c >> (1 + a)) & 1) != bool(flip[r])
            out[r, 1 + a] = -y[r, 1 + k] if neg else y[r, 1 + k]
    return out


def surrogate_class(spec, nbr, phi32, ties=False):
    """Classes (0 in, 1 out, 2 fallback, 3 network; 255 far) of the float
    field phi32, decided on its real values in double precision.  With
    ties=True also returns the number of points whose |kappa| h lies within
    1e-9 (relative) of the 0.1 bound."""
    phi32 = np.ascontiguousarray(phi32, np.float32)
    P = phi32.shape[0]
    cls = np.empty((P, 64), np.uint8)
    nt = C.c_int64(0)
    lib().or_surrogate_class(C.byref(_grid(spec)), C.c_int64(P), _p(np.ascontiguousarray(nbr, np.int32)),
                             _p(phi32), _p(cls), C.byref(nt))
    return (cls, int(nt.value)) if ties else cls


def coarser(spec):
    """The layer below spec: same lo, half the dims, twice the spacing."""
    import sg_inputs as si
    assert all(int(d) % 2 == 0 for d in spec.dims)
    return si.GridSpec(tuple(spec.lo), tuple(int(d) // 2 for d in spec.dims), 2.0 * spec.h,
                       kernel_support=2.0 * spec.kernel_support, heaviside_eps=2.0 * spec.heaviside_eps,
                       id_order=spec.id_order)


def build_layers(spec, shape, layers):
    """Multi-resolution stack, coarsest first: layer 0 tagged in full, every
    finer layer tagged from the one below it.  Returns a list of namespaces
    (as build_grid, plus `evaluated`)."""
    specs = [spec]
    for _ in range(layers - 1):
        specs.append(coarser(specs[-1]))
    specs.reverse()
    out = [build_grid(specs[0], shape)]
    out[0].evaluated = specs[0].n_cells
    for sp in specs[1:]:
        c = out[-1]
        cell_pkg, cell_type, P, ties, ev = tag_from(sp, shape, c.spec, c.cell_pkg, c.pkg_type, c.phi)
        pkg_cell, pkg_type, nbr = tables(sp, cell_pkg, cell_type, P)
        phi = init_sdf(sp, shape, P, pkg_cell)
        out.append(types.SimpleNamespace(spec=sp, shape=shape, P=P, near_ties=ties, cell_pkg=cell_pkg,
                                         cell_type=cell_type, pkg_cell=pkg_cell, pkg_type=pkg_type, nbr=nbr,
                                         phi=phi, evaluated=ev))
    return out


def build_grid(spec, shape, far=None):
    """Tag, allocate, build tables and initialise phi.  Returns a namespace."""
    cell_pkg, cell_type, P, ties = tag(spec, shape)
    pkg_cell, pkg_type, nbr = tables(spec, cell_pkg, cell_type, P)
    phi = init_sdf(spec, shape, P, pkg_cell, far)
    return types.SimpleNamespace(spec=spec, shape=shape, P=P, near_ties=ties, cell_pkg=cell_pkg,
                                 cell_type=cell_type, pkg_cell=pkg_cell, pkg_type=pkg_type, nbr=nbr, phi=phi)
