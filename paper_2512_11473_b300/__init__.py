"""Python binding of libsg, the sm_103a CUDA library for contiguous sparse-grid
level sets (Gu & Hu, "Contiguous Storage of Grid Data for Heterogeneous
Computing").

Argument marshalling only: every step runs in the library's kernels.  PyTorch
supplies device memory (the caching allocator, through the library's
allocator hook), the current CUDA stream, and tensor views of the library's
device arrays.  There is no CPU fallback: without ``libsg.so`` or a CUDA
device the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsg.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "sg.h")

(SG_OK, SG_ERR_INVALID, SG_ERR_OOM, SG_ERR_CUDA, SG_ERR_STATE, SG_ERR_CAPACITY, SG_ERR_TIMEOUT, SG_ERR_DEVICE,
 SG_ERR_IO) = range(9)
STATUS_NAMES = ["SG_OK", "SG_ERR_INVALID", "SG_ERR_OOM", "SG_ERR_CUDA", "SG_ERR_STATE", "SG_ERR_CAPACITY",
                "SG_ERR_TIMEOUT", "SG_ERR_DEVICE", "SG_ERR_IO"]

FIELDS = {"phi": 0, "gx": 1, "gy": 2, "gz": 3, "W": 4, "Gx": 5, "Gy": 6, "Gz": 7, "lap": 8, "S0": 9}
INT_FIELDS = {"cell_pkg": (100, "<i4"), "pkg_cell": (101, "<i4"), "pkg_type": (102, "|u1"), "nbr": (103, "<i4")}
PROBE_MORTON = 1
DEBUG_CC_ABSENT_POINTS, DEBUG_CC_ABSENT_CELLS, DEBUG_CC_PER_SWEEP = 1, 2, 4
PROBE_OUTPUTS = ("phi", "nx", "ny", "nz", "W", "Gx", "Gy", "Gz")


class SgError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("%s: %s" % (name, msg))


class sg_shape(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad", C.c_int32), ("centre", C.c_double * 3), ("rot", C.c_double * 9),
                ("p", C.c_double * 8)]


class sg_grid_desc(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("dims", C.c_int32 * 3), ("id_order", C.c_int32), ("h", C.c_double),
                ("far_value", C.c_double), ("kernel_support", C.c_double), ("heaviside_eps", C.c_double)]


class sg_batch_plan(C.Structure):
    _fields_ = [("pkgs_per_item", C.c_int32), ("depth", C.c_int32), ("reinit_iterations", C.c_int32),
                ("cfl", C.c_float), ("integrals_mode", C.c_int32), ("reserved", C.c_int32)]


class sg_relax(C.Structure):
    _fields_ = [("n", C.c_int64), ("offsets", C.POINTER(C.c_int64)), ("x", C.c_void_p), ("y", C.c_void_p),
                ("z", C.c_void_p), ("out", C.c_void_p * 8), ("steps", C.c_int32), ("step", C.c_float),
                ("sweeps", C.c_int32), ("reserved", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class sg_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


def declared_symbols(header=HEADER):
    """Names of the functions the public header declares."""
    text = open(header).read()
    return re.findall(r"^SG_API\s+[\w\s\*]+?\b(sg_\w+)\s*\(", text, flags=re.M)


_lib = None


def lib():
    """Load libsg.so (raises when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libsg.so not built: run `python -m paper_2512_11473_b300.build` "
                              "(or __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        L.sg_create.argtypes = [C.POINTER(sg_grid_desc), C.POINTER(sg_allocator), vp, C.POINTER(vp)]
        L.sg_destroy.argtypes = [vp]
        L.sg_tag_allocate.argtypes = [vp, C.POINTER(sg_shape), C.POINTER(i64)]
        L.sg_init_sdf.argtypes = [vp, C.POINTER(sg_shape)]
        L.sg_gradient.argtypes = [vp]
        L.sg_laplacian.argtypes = [vp]
        L.sg_sequential_update.argtypes = [vp, C.c_float]
        L.sg_consistency_correct.argtypes = [vp, C.c_float, C.POINTER(i64)]
        L.sg_debug_consistency_absent_cta.argtypes = [vp, C.c_float]
        L.sg_debug_wide_offsets.argtypes = [C.c_int32]
        L.sg_debug_wide_offsets.restype = None
        L.sg_debug_consistency.argtypes = [vp, C.c_float, C.c_int32, C.POINTER(i64)]
        L.sg_tag_allocate_from.argtypes = [vp, vp, C.POINTER(sg_shape), C.POINTER(i64), C.POINTER(i64)]
        L.sg_multires_layers.argtypes = [C.POINTER(sg_grid_desc), i32]
        L.sg_multires_layers.restype = i32
        L.sg_reinit.argtypes = [vp, i32, C.c_float]
        L.sg_kernel_integrals.argtypes = [vp, i32, vp]
        L.sg_probe.argtypes = [vp, i64, vp, vp, vp] + [vp] * 8 + [i32]
        L.sg_morton_order.argtypes = [vp, i64, vp, vp, vp, vp, vp]
        L.sg_morton_order_noalloc.argtypes = [C.POINTER(sg_grid_desc), i64, vp, vp, vp, vp, vp, vp]
        L.sg_get_field.argtypes = [vp, i32, C.POINTER(vp), C.POINTER(i64)]
        L.sg_n_packages.argtypes = [vp]
        L.sg_n_packages.restype = i64
        L.sg_set_stream.argtypes = [vp, vp]
        L.sg_check_tables.argtypes = [vp]
        L.sg_restore.argtypes = [vp, i64, vp, vp, vp, vp, vp]
        L.sg_clear_error.argtypes = [vp]
        L.sg_status_sync.argtypes = [vp]
        L.sg_last_error.argtypes = [vp]
        L.sg_last_error.restype = C.c_char_p
        L.sg_version.restype = C.c_char_p
        L.sg_kernel_launch_count.restype = i64
        L.sg_mlp_create.argtypes = [vp, vp, C.POINTER(vp)]
        L.sg_mlp_destroy.argtypes = [vp]
        L.sg_mlp_set_params.argtypes = [vp, vp]
        L.sg_mlp_get_params.argtypes = [vp, vp]
        L.sg_mlp_forward.argtypes = [vp, i64, vp, vp]
        L.sg_mlp_loss_grad.argtypes = [vp, i64, vp, vp, vp, vp, vp]
        L.sg_mlp_train_step.argtypes = [vp, i64, vp, vp, vp, C.c_float, vp]
        L.sg_mlp_last_error.argtypes = [vp]
        L.sg_mlp_last_error.restype = C.c_char_p
        L.sg_surrogate_classify.argtypes = [vp, vp]
        L.sg_surrogate_samples.argtypes = [vp, C.c_uint64, C.c_float, i64, vp, vp, C.POINTER(i64)]
        L.sg_surrogate_stats.argtypes = [vp, C.POINTER(i64)]
        L.sg_batch_create.argtypes = [C.POINTER(vp), i32, vp, C.POINTER(vp)]
        L.sg_batch_destroy.argtypes = [vp]
        L.sg_batch_reset.argtypes = [vp]
        L.sg_batch_run.argtypes = [vp, C.POINTER(sg_batch_plan)]
        L.sg_batch_autotune.argtypes = [vp, C.POINTER(sg_batch_plan), i32, C.POINTER(C.c_float)]
        L.sg_batch_autotune_cached.argtypes = [vp, C.POINTER(sg_batch_plan), i32, C.c_char_p, C.POINTER(i32)]
        L.sg_batch_autotune_key.argtypes = [vp, C.POINTER(sg_batch_plan), C.c_char_p, i32]
        L.sg_autotune_cache_lookup.argtypes = [C.c_char_p, C.c_char_p, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
        L.sg_autotune_cache_store.argtypes = [C.c_char_p, C.c_char_p, i32, i32]
        L.sg_batch_get_field.argtypes = [vp, i32, i32, C.POINTER(vp), C.POINTER(i64)]
        L.sg_batch_n_packages.argtypes = [vp]
        L.sg_batch_n_packages.restype = i64
        L.sg_batch_last_error.argtypes = [vp]
        L.sg_batch_set_surrogate.argtypes = [vp, vp]
        L.sg_batch_relax.argtypes = [vp, C.POINTER(sg_batch_plan), C.POINTER(sg_relax)]
        L.sg_batch_last_error.restype = C.c_char_p
        for name in declared_symbols():
            f = getattr(L, name)
            if f.restype is C.c_int:  # default: sg_status
                f.restype = i32
        _lib = L
    return _lib


def _torch():
    import torch
    return torch


class _CudaArray:
    """Minimal __cuda_array_interface__ holder for zero-copy tensor views."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def _as_shape(s) -> sg_shape:
    out = sg_shape()
    out.kind = int(s.kind)
    out.centre[:] = [float(v) for v in s.centre]
    out.rot[:] = [float(v) for v in s.rot]
    out.p[:] = [float(v) for v in s.p]
    return out


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


class _TorchAllocator:
    """Routes the library's allocations through torch's caching allocator."""

    def __init__(self, device):
        torch = _torch()
        self.device = device

        def _alloc(nbytes, stream, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), device=self.device, stream=stream or 0)
            except Exception:  # out of memory: the library reports SG_ERR_OOM
                return None

        def _free(ptr, nbytes, stream, ctx):
            torch.cuda.caching_allocator_delete(ptr)

        self.alloc_fn = ALLOC_FN(_alloc)
        self.free_fn = FREE_FN(_free)
        self.struct = sg_allocator(self.alloc_fn, self.free_fn, None)


class Grid:
    """A sparse narrow-band grid on one CUDA device.

    ``spec`` needs ``lo`` (3 floats), ``dims`` (3 ints) and ``h``, and may set
    ``kernel_support``, ``heaviside_eps`` and ``id_order`` (see sg_grid_desc).
    Calls are queued on ``stream`` (default: torch's current stream at
    construction).
    """

    def __init__(self, spec, far_value=0.0, stream=None, torch_allocator=True, allocator=None):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2512_11473_b300 needs a CUDA device")
        self._lib = lib()
        self.device = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.spec = spec
        d = _desc(spec, far_value)
        # allocator: any object with an sg_allocator ``struct`` (kept alive here)
        self._alloc = allocator if allocator is not None else (_TorchAllocator(self.device) if torch_allocator else None)
        h = C.c_void_p()
        st = self._lib.sg_create(C.byref(d), C.byref(self._alloc.struct) if self._alloc else None,
                                 C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != SG_OK:
            raise SgError(st, "sg_create failed")
        self._h = h
        self.P = 0

    # -- plumbing ------------------------------------------------------------
    def _check(self, st):
        if st != SG_OK:
            raise SgError(st, self._lib.sg_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    def set_stream(self, stream):
        self.stream = stream
        self._check(self._lib.sg_set_stream(self._h, C.c_void_p(stream.cuda_stream)))

    def sync(self):
        """Synchronise the stream; raise on a sticky device error."""
        self._check(self._lib.sg_status_sync(self._h))

    def check_tables(self):
        """Queue the device check of the cell, package, neighbour and face
        tables; a later sync() raises if they disagree."""
        self._check(self._lib.sg_check_tables(self._h))

    def clear_error(self):
        self._check(self._lib.sg_clear_error(self._h))

    # -- the hot path --------------------------------------------------------
    def tag_allocate(self, shape) -> int:
        n = C.c_int64(0)
        self._check(self._lib.sg_tag_allocate(self._h, C.byref(_as_shape(shape)), C.byref(n)))
        self.P = int(n.value)
        return self.P

    def tag_allocate_from(self, coarse, shape):
        """Tag this layer from its coarser layer (see sg_tag_allocate_from).
        Returns (P, cells whose distance was evaluated)."""
        n, ev = C.c_int64(0), C.c_int64(0)
        self._check(self._lib.sg_tag_allocate_from(self._h, coarse.handle, C.byref(_as_shape(shape)), C.byref(n),
                                                   C.byref(ev)))
        self.P = int(n.value)
        return self.P, int(ev.value)

    def init_sdf(self, shape):
        self._check(self._lib.sg_init_sdf(self._h, C.byref(_as_shape(shape))))

    def gradient(self):
        self._check(self._lib.sg_gradient(self._h))

    def laplacian(self):
        self._check(self._lib.sg_laplacian(self._h))

    def consistency_correct(self, trust=1.0):
        """Sign correction of phi and of the far cells (trust band |phi| <
        trust h).  Returns (points flipped, far cells moved, point sweeps,
        cell sweeps)."""
        out = (C.c_int64 * 4)()
        self._check(self._lib.sg_consistency_correct(self._h, float(trust), out))
        return tuple(int(v) for v in out)

    def debug_consistency_absent_cta(self, trust=1.0):
        """Testing hook: the correction with a CTA that never reaches the
        floods' grid barriers; raises SgError (SG_ERR_TIMEOUT) once the
        bounded waits give up, with phi and the tables unchanged."""
        self._check(self._lib.sg_debug_consistency_absent_cta(self._h, float(trust)))

    def debug_consistency(self, trust=1.0, flags=0):
        """Testing hook: the correction with SG_DEBUG_CC_* flags (an absent CTA
        in the point or cell flood, or the per-sweep floods).  Returns the
        counts as consistency_correct."""
        out = (C.c_int64 * 4)()
        self._check(self._lib.sg_debug_consistency(self._h, float(trust), int(flags), out))
        return tuple(int(v) for v in out)

    def sequential_update(self, delta):
        """phi <- phi + delta on every active value (the paper's sequential benchmark)."""
        self._check(self._lib.sg_sequential_update(self._h, float(delta)))

    def reinit(self, iterations, cfl=0.5):
        self._check(self._lib.sg_reinit(self._h, int(iterations), float(cfl)))

    def kernel_integrals(self, mode=0, mlp=None):
        """mode 0: exact; mode 1: surrogate network `mlp` (an MLP) with exact fallback."""
        self._check(self._lib.sg_kernel_integrals(self._h, int(mode), mlp.handle if mlp is not None else None))

    def surrogate_classify(self):
        torch = _torch()
        cls = torch.empty(self.n_packages() * 64, dtype=torch.uint8, device="cuda")
        self._check(self._lib.sg_surrogate_classify(self._h, _ptr(cls)))
        return cls.view(-1, 64)

    def surrogate_samples(self, seed, keep=1.0, cap=None):
        """(x bf16 [n, 32], t float32 [n, 4], selected count) of this grid's
        network-class points; needs current exact integrals."""
        torch = _torch()
        n = C.c_int64()
        if cap is None:
            self._check(self._lib.sg_surrogate_samples(self._h, seed, float(keep), 0, None, None, C.byref(n)))
            cap = n.value
        x = torch.empty((max(cap, 1), 32), dtype=torch.bfloat16, device="cuda")
        t = torch.empty((max(cap, 1), 4), dtype=torch.float32, device="cuda")
        self._check(self._lib.sg_surrogate_samples(self._h, seed, float(keep), int(cap), _ptr(x), _ptr(t),
                                                   C.byref(n)))
        m = min(cap, n.value)
        return x[:m], t[:m], n.value

    def surrogate_stats(self):
        """Points per class (in, out, fallback, network) of the last mode-1 call."""
        c = (C.c_int64 * 4)()
        self._check(self._lib.sg_surrogate_stats(self._h, c))
        return [int(v) for v in c]

    def probe(self, x, y, z, morton=True, out=None, outputs=PROBE_OUTPUTS):
        """Probe at device float32 tensors x, y, z; returns a dict of outputs.

        ``out`` may supply preallocated device tensors (dict by name)."""
        torch = _torch()
        n = x.numel()
        res = {}
        for name in PROBE_OUTPUTS:
            if name in outputs:
                res[name] = out[name] if out is not None else torch.empty(n, dtype=torch.float32, device=x.device)
        ptrs = [_ptr(res.get(name)) for name in PROBE_OUTPUTS]
        self._check(self._lib.sg_probe(self._h, n, _ptr(x), _ptr(y), _ptr(z), *ptrs,
                                       PROBE_MORTON if morton else 0))
        return res

    def morton_order(self, x, y, z):
        torch = _torch()
        n = x.numel()
        keys = torch.empty(n, dtype=torch.int64, device=x.device)
        order = torch.empty(n, dtype=torch.int32, device=x.device)
        self._check(self._lib.sg_morton_order(self._h, n, _ptr(x), _ptr(y), _ptr(z), _ptr(keys), _ptr(order)))
        return keys, order

    # -- views ---------------------------------------------------------------
    def field(self, name):
        """Borrowed zero-copy tensor view of a device array of the grid."""
        torch = _torch()
        p = C.c_void_p()
        n = C.c_int64()
        if name in FIELDS:
            self._check(self._lib.sg_get_field(self._h, FIELDS[name], C.byref(p), C.byref(n)))
            t = torch.as_tensor(_CudaArray(p.value, (n.value,), "<f4"), device="cuda")
            return t.view(-1, 64)
        fid, typestr = INT_FIELDS[name]
        self._check(self._lib.sg_get_field(self._h, fid, C.byref(p), C.byref(n)))
        t = torch.as_tensor(_CudaArray(p.value, (n.value,), typestr), device="cuda")
        return t.view(-1, 27) if name == "nbr" else t

    def n_packages(self) -> int:
        return int(self._lib.sg_n_packages(self._h))

    # -- checkpoint ------------------------------------------------------------
    def checkpoint(self, fields=("phi", "gx", "gy", "gz", "W", "Gx", "Gy", "Gz")):
        """Host copy of the grid: the tagging's tables and the named float
        fields (numpy arrays), for save_checkpoint / restore."""
        ck = {"P": np.int64(self.P)}
        for name in ("cell_pkg", "pkg_cell", "pkg_type", "nbr"):
            ck[name] = self.field(name).cpu().numpy().copy()
        for name in fields:
            ck[name] = self.field(name).cpu().numpy().copy()
        return ck

    def restore(self, ck):
        """Put a checkpoint back (a grid created with the same description):
        tables and phi through sg_restore (checked), the other fields through
        their device views."""
        torch = _torch()
        arrs = {k: np.ascontiguousarray(ck[k]) for k in ("cell_pkg", "pkg_cell", "pkg_type", "nbr")}
        assert arrs["cell_pkg"].dtype == np.int32 and arrs["nbr"].dtype == np.int32
        phi = np.ascontiguousarray(ck["phi"], np.float32) if "phi" in ck else None
        self._check(self._lib.sg_restore(self._h, int(ck["P"]), *(arrs[k].ctypes.data_as(C.c_void_p)
                                                                 for k in ("cell_pkg", "pkg_cell", "pkg_type", "nbr")),
                                         phi.ctypes.data_as(C.c_void_p) if phi is not None else None))
        self.P = int(ck["P"])
        for name in FIELDS:
            if name != "phi" and name in ck:
                self.field(name).copy_(torch.from_numpy(np.ascontiguousarray(ck[name], np.float32)))
        torch.cuda.synchronize()


BATCH_CANDIDATES = ((1, 1), (2, 1), (2, 2), (4, 1), (4, 2), (8, 1), (8, 2))


def make_plan(pkgs_per_item=4, depth=2, reinit_iterations=20, cfl=0.5, integrals_mode=0) -> sg_batch_plan:
    return sg_batch_plan(int(pkgs_per_item), int(depth), int(reinit_iterations), float(cfl), int(integrals_mode), 0)


class Batch:
    """Many initialised grids swept together (one persistent launch per
    sweep, the sequence captured as a CUDA graph).  The grids' phi is copied
    at construction."""

    def __init__(self, grids, stream=None):
        torch = _torch()
        self._lib = lib()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.n = len(grids)
        arr = (C.c_void_p * self.n)(*[g.handle.value for g in grids])
        h = C.c_void_p()
        st = self._lib.sg_batch_create(arr, self.n, C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != SG_OK:
            raise SgError(st, "sg_batch_create failed")
        self._h = h
        self.P = int(self._lib.sg_batch_n_packages(h))

    def _check(self, st):
        if st != SG_OK:
            raise SgError(st, self._lib.sg_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        self._check(self._lib.sg_batch_reset(self._h))

    def run(self, plan=None, **kw):
        plan = plan if plan is not None else make_plan(**kw)
        self._check(self._lib.sg_batch_run(self._h, C.byref(plan)))
        return plan

    def autotune(self, plan=None, reps=3, **kw):
        """Returns (best plan, {(pkgs_per_item, depth): ms})."""
        plan = plan if plan is not None else make_plan(**kw)
        times = (C.c_float * 8)()
        self._check(self._lib.sg_batch_autotune(self._h, C.byref(plan), int(reps), times))
        return plan, {c: float(times[i]) for i, c in enumerate(BATCH_CANDIDATES)}

    def autotune_cached(self, path, plan=None, reps=3, **kw):
        """sg_batch_autotune_cached: returns (plan, hit), hit True when the
        cache file `path` already held this batch's key."""
        plan = plan if plan is not None else make_plan(**kw)
        hit = C.c_int32(0)
        self._check(self._lib.sg_batch_autotune_cached(self._h, C.byref(plan), int(reps), os.fsencode(path),
                                                       C.byref(hit)))
        return plan, bool(hit.value)

    def autotune_key(self, plan=None, **kw):
        plan = plan if plan is not None else make_plan(**kw)
        buf = C.create_string_buffer(400)
        self._check(self._lib.sg_batch_autotune_key(self._h, C.byref(plan), buf, 400))
        return buf.value.decode()

    def field(self, body, name):
        torch = _torch()
        p = C.c_void_p()
        n = C.c_int64()
        if name in ("nbr", "cell_pkg"):
            self._check(self._lib.sg_batch_get_field(self._h, int(body), INT_FIELDS[name][0], C.byref(p), C.byref(n)))
            t = torch.as_tensor(_CudaArray(p.value, (n.value,), "<i4"), device="cuda")
            return t.view(-1, 27) if name == "nbr" else t
        self._check(self._lib.sg_batch_get_field(self._h, int(body), FIELDS[name], C.byref(p), C.byref(n)))
        return torch.as_tensor(_CudaArray(p.value, (n.value,), "<f4"), device="cuda").view(-1, 64)

    def set_surrogate(self, mlp):
        """Bind the network of plans with integrals_mode=1 (None unbinds)."""
        self._mlp = mlp  # the batch borrows it
        self._check(self._lib.sg_batch_set_surrogate(self._h, mlp.handle if mlp is not None else None))

    def relax(self, x, y, z, offsets, steps, step=0.1, plan=None, sweeps=True, out=None):
        """[The plan's sweeps, then] `steps` relaxation steps of the particles
        (x, y, z: float32 CUDA tensors updated in place, stored body after body,
        body i owning [offsets[i], offsets[i+1])).  out: dict of the probe
        outputs (names of PROBE_OUTPUTS) the last step writes."""
        n = int(x.numel())
        for v in (x, y, z):
            assert v.dtype == _torch().float32 and v.is_cuda and v.is_contiguous() and v.numel() == n
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        assert off.size == self.n + 1
        r = sg_relax()
        r.n = n
        self._relax_offsets = off  # kept alive for the call
        r.offsets = off.ctypes.data_as(C.POINTER(C.c_int64))
        r.x, r.y, r.z = x.data_ptr(), y.data_ptr(), z.data_ptr()
        out = out or {}
        for i, name in enumerate(PROBE_OUTPUTS):
            t = out.get(name)
            if t is not None:
                assert t.dtype == _torch().float32 and t.is_cuda and t.is_contiguous() and t.numel() == n
            r.out[i] = t.data_ptr() if t is not None else None
        r.steps = int(steps)
        r.step = float(step)
        r.sweeps = 1 if sweeps else 0
        if sweeps:
            plan = plan if plan is not None else make_plan()
            self._check(self._lib.sg_batch_relax(self._h, C.byref(plan), C.byref(r)))
        else:
            self._check(self._lib.sg_batch_relax(self._h, None, C.byref(r)))
        return plan


MLP_NPARAM = 6212
SUR_CLASSES = ("trivial_in", "trivial_out", "fallback", "network")


class MLP:
    """The kernel-integral surrogate network on the current device."""

    def __init__(self, params, stream=None):
        torch = _torch()
        self._lib = lib()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == MLP_NPARAM
        h = C.c_void_p()
        st = self._lib.sg_mlp_create(p.ctypes.data_as(C.c_void_p), C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != SG_OK:
            raise SgError(st, "sg_mlp_create failed")
        self._h = h

    @property
    def handle(self):
        return self._h

    def _check(self, st):
        if st != SG_OK:
            raise SgError(st, self._lib.sg_mlp_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sg_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        self._check(self._lib.sg_mlp_set_params(self._h, p.ctypes.data_as(C.c_void_p)))

    def get_params(self):
        p = np.empty(MLP_NPARAM, np.float32)
        self._check(self._lib.sg_mlp_get_params(self._h, p.ctypes.data_as(C.c_void_p)))
        return p

    def forward(self, x):
        torch = _torch()
        y = torch.empty((x.shape[0], 4), dtype=torch.float32, device=x.device)
        self._check(self._lib.sg_mlp_forward(self._h, x.shape[0], _ptr(x), _ptr(y)))
        return y

    def loss_grad(self, x, t, idx=None):
        torch = _torch()
        n = idx.numel() if idx is not None else x.shape[0]
        g = torch.empty(MLP_NPARAM, dtype=torch.float32, device=x.device)
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
        self._check(self._lib.sg_mlp_loss_grad(self._h, n, _ptr(x), _ptr(t), _ptr(idx), _ptr(g), _ptr(loss)))
        return g, loss

    def train_step(self, x, t, idx, lr, loss=None):
        n = idx.numel() if idx is not None else x.shape[0]
        self._check(self._lib.sg_mlp_train_step(self._h, n, _ptr(x), _ptr(t), _ptr(idx), float(lr), _ptr(loss)))


NOALLOC_MAX_PARTICLES = 262144


def _desc(spec, far_value=0.0) -> sg_grid_desc:
    d = sg_grid_desc()
    d.lo[:] = [float(v) for v in spec.lo]
    d.dims[:] = [int(v) for v in spec.dims]
    d.h = float(spec.h)
    d.far_value = float(far_value)
    d.id_order = int(getattr(spec, "id_order", 0) or 0)
    d.kernel_support = float(getattr(spec, "kernel_support", 0.0) or 0.0)
    d.heaviside_eps = float(getattr(spec, "heaviside_eps", 0.0) or 0.0)
    return d


def multires_layers(spec, min_dims=8) -> int:
    """Layer count of a multi-resolution stack ending at spec (sg_multires_layers)."""
    return int(lib().sg_multires_layers(C.byref(_desc(spec)), int(min_dims)))


def layer_spec(spec, level, layers):
    """Grid spec of layer `level` (0 coarsest) of a stack of `layers` ending at spec."""
    import sg_inputs as si
    k = layers - 1 - level
    f = 1 << k
    assert all(int(d) % f == 0 for d in spec.dims)
    # the options keep their meaning relative to each layer's spacing
    return si.GridSpec(tuple(spec.lo), tuple(int(d) // f for d in spec.dims), spec.h * f,
                       kernel_support=spec.kernel_support * f, heaviside_eps=spec.heaviside_eps * f,
                       id_order=spec.id_order)


class MultiResolution:
    """A stack of grids over one domain, each doubling the resolution of the
    one below ("Multi-resolution Level-set"): the coarsest layer is tagged in
    full, every finer layer from the layer below it; each is initialised.
    layers defaults to multires_layers(spec, min_dims)."""

    def __init__(self, spec, shape, layers=None, min_dims=8, stream=None):
        self.layers = int(layers) if layers else multires_layers(spec, min_dims)
        self.grids, self.evaluated = [], []
        for k in range(self.layers):
            g = Grid(layer_spec(spec, k, self.layers), stream=stream)
            if k == 0:
                g.tag_allocate(shape)
                ev = g.spec.n_cells
            else:
                _, ev = g.tag_allocate_from(self.grids[-1], shape)
            g.init_sdf(shape)
            self.grids.append(g)
            self.evaluated.append(int(ev))

    @property
    def finest(self):
        return self.grids[-1]

    def close(self):
        for g in self.grids:
            g.close()
        self.grids = []


def save_checkpoint(path, grid=None, mlp=None):
    """One .npz file with a grid's checkpoint (Grid.checkpoint) and/or a
    network's parameters: the FP32 master vector and its BF16 rounding (the
    values the tensor cores use), as raw arrays."""
    out = {}
    if grid is not None:
        out.update({"grid_" + k: v for k, v in grid.checkpoint().items()})
    if mlp is not None:
        par = mlp.get_params()
        out["mlp_master"] = par
        out["mlp_bf16"] = (par.view(np.uint32) + 0x7FFF + ((par.view(np.uint32) >> 16) & 1) >> 16).astype(np.uint16)
    np.savez(path, **out)


def load_checkpoint(path, grid=None, mlp=None):
    """Restore what save_checkpoint wrote into a grid (of the same
    description) and/or a network."""
    d = np.load(path)
    if grid is not None:
        grid.restore({k[5:]: d[k] for k in d.files if k.startswith("grid_")})
    if mlp is not None:
        mlp.set_params(d["mlp_master"])


def morton_order_noalloc(spec, x, y, z, keys=None, order=None, stream=None):
    """Morton keys and order through the allocation-free entry point.

    For callers whose device memory is not the library's to take: the library
    allocates nothing here and uses its built-in scratch (at most
    NOALLOC_MAX_PARTICLES particles).  ``x``, ``y``, ``z`` are contiguous
    float32 CUDA tensors of one length on one device; ``keys`` / ``order`` may
    be caller tensors (contiguous int64 / int32 of at least that length on the
    same device); otherwise they are created here by torch on the caller's
    behalf.  The call runs with x's device current, on ``stream`` (default:
    that device's current stream)."""
    torch = _torch()
    n = x.numel()
    dev = x.device
    for name, t in (("x", x), ("y", y), ("z", z)):
        if not (t.is_cuda and t.device == dev and t.dtype == torch.float32 and t.is_contiguous() and t.numel() == n):
            raise ValueError("%s: contiguous float32 CUDA tensor of %d values on %s expected" % (name, n, dev))
    if keys is None:
        keys = torch.empty(n, dtype=torch.int64, device=dev)
    if order is None:
        order = torch.empty(n, dtype=torch.int32, device=dev)
    for name, t, dt in (("keys", keys, torch.int64), ("order", order, torch.int32)):
        if not (t.is_cuda and t.device == dev and t.dtype == dt and t.is_contiguous() and t.numel() >= n):
            raise ValueError("%s: contiguous %s CUDA tensor of >= %d values on %s expected" % (name, dt, n, dev))
    with torch.cuda.device(dev):
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        st = lib().sg_morton_order_noalloc(C.byref(_desc(spec)), n, _ptr(x), _ptr(y), _ptr(z), _ptr(keys),
                                           _ptr(order), C.c_void_p(s.cuda_stream))
    if st != SG_OK:
        raise SgError(st, "sg_morton_order_noalloc failed")
    return keys, order


def autotune_cache_lookup(path, key):
    """(pkgs_per_item, depth) of key's entry in an autotuner cache file, or
    None (sg_autotune_cache_lookup; host only)."""
    ppi, dep, found = C.c_int32(0), C.c_int32(0), C.c_int32(0)
    st = lib().sg_autotune_cache_lookup(os.fsencode(path), key.encode(), C.byref(ppi), C.byref(dep), C.byref(found))
    if st != SG_OK:
        raise SgError(st, "sg_autotune_cache_lookup failed")
    return (ppi.value, dep.value) if found.value else None


def autotune_cache_store(path, key, pkgs_per_item, depth):
    """Append an entry to an autotuner cache file (sg_autotune_cache_store; host only)."""
    st = lib().sg_autotune_cache_store(os.fsencode(path), key.encode(), int(pkgs_per_item), int(depth))
    if st != SG_OK:
        raise SgError(st, "sg_autotune_cache_store failed")


def version() -> str:
    return lib().sg_version().decode()


def kernel_launch_count() -> int:
    """Kernels launched by libsg in this process so far."""
    return int(lib().sg_kernel_launch_count())


def debug_wide_offsets(on: bool) -> None:
    """Testing hook (process-wide): take the 64-bit address kernels of the
    probe, the exact integrals and the relaxation at any store size (see
    sg_debug_wide_offsets); results are bitwise the same."""
    lib().sg_debug_wide_offsets(1 if on else 0)
