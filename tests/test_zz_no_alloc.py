"""The allocation-free Morton-order entry point against the regular one.

sg_morton_order_noalloc serves callers that cannot let the library allocate
device memory (their memory belongs to their own pool, or they cannot take
the device-wide synchronisation of cudaMalloc/cudaFree).  Its scratch is a
static device array shared by every call, so the test makes two calls in a
row with different sizes and key widths and compares each with
sg_morton_order on a grid: keys and order must agree bit for bit.  This file
is collected last so that a failure here leaves every other test already run.
"""
import ctypes as C
import gc

import numpy as np
import pytest

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


def _regular(sg, spec, shape, X, Y, Z):
    g = sg.Grid(spec)
    g.tag_allocate(shape)
    keys, order = g.morton_order(X, Y, Z)
    torch.cuda.synchronize()
    return keys.cpu(), order.cpu()


def _noalloc_raw(sg, spec, X, Y, Z, check_free=False):
    """Direct C-ABI call with caller-owned outputs.  check_free: the device's
    free memory (cudaMemGetInfo) must not drop across the call, which catches
    a cudaMalloc by the library as well as an allocation through torch (the
    first call on a device may load the library's module and its static
    scratch array, so only a later call is checked)."""
    n = X.numel()
    keys = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    order = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    desc = sg._desc(spec)
    args = [C.c_void_p(t.data_ptr()) for t in (X, Y, Z, keys, order)]
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    # objects of earlier tests may still be waiting for the collector; their
    # finalizers free memory, so collect first and keep the collector off
    gc.collect()
    gc.disable()
    try:
        torch.cuda.synchronize()
        before = torch.cuda.memory_allocated()
        free0 = torch.cuda.mem_get_info()[0]
        st = sg.lib().sg_morton_order_noalloc(C.byref(desc), n, *args[:3], *args[3:], stream)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        after = torch.cuda.memory_allocated()
    finally:
        gc.enable()
    assert st == sg.SG_OK
    assert after <= before
    if check_free:
        assert free1 >= free0
    return keys.cpu(), order.cpu()


def test_noalloc_matches_regular_entry_point_twice(sg):
    # call 1: 32-bit keys, 200,000 particles
    shape1 = si.torus(0.6, 0.2)
    spec1 = si.GridSpec((-1.0, -1.0, -0.4), (50, 50, 20), 0.01)
    x, y, z = si.box_particles(200_000, np.array(spec1.lo) - 0.05, np.array(spec1.hi()) + 0.05, seed=31)
    X1, Y1, Z1 = (torch.from_numpy(v).cuda() for v in (x, y, z))
    # call 2: 64-bit keys, fewer particles, so stale scratch from call 1 would show
    shape2 = si.sphere(0.004)
    spec2 = si.GridSpec((-1.0, -1.0, -1.0), (600, 3, 3), 2.0 / 2400)
    x, y, z = si.box_particles(70_001, spec2.lo, spec2.hi(), seed=32)
    x[10:20] = x[0]
    y[10:20] = y[0]
    z[10:20] = z[0]
    X2, Y2, Z2 = (torch.from_numpy(v).cuda() for v in (x, y, z))

    got1 = _noalloc_raw(sg, spec1, X1, Y1, Z1)
    got2 = _noalloc_raw(sg, spec2, X2, Y2, Z2, check_free=True)
    ref1 = _regular(sg, spec1, shape1, X1, Y1, Z1)
    ref2 = _regular(sg, spec2, shape2, X2, Y2, Z2)
    assert torch.equal(got1[0], ref1[0]) and torch.equal(got1[1], ref1[1])
    assert torch.equal(got2[0], ref2[0]) and torch.equal(got2[1], ref2[1])
    assert int(ref2[0].max()) >= 2 ** 32  # the second call used the 64-bit sort
    # the binding's wrapper goes through the same entry point
    k, o = sg.morton_order_noalloc(spec1, X1, Y1, Z1)
    assert torch.equal(k.cpu(), ref1[0]) and torch.equal(o.cpu(), ref1[1])


def test_noalloc_limits(sg):
    spec = si.GridSpec((-1.0, -1.0, -0.4), (50, 50, 20), 0.01)
    n = sg.NOALLOC_MAX_PARTICLES
    X = torch.zeros(n + 1, device="cuda")
    with pytest.raises(sg.SgError) as e:
        sg.morton_order_noalloc(spec, X, X, X)
    assert e.value.status == sg.SG_ERR_CAPACITY
    # exactly at the limit is accepted and matches the regular path
    x, y, z = si.box_particles(n, spec.lo, spec.hi(), seed=33)
    Xs = [torch.from_numpy(v).cuda() for v in (x, y, z)]
    k, o = sg.morton_order_noalloc(spec, *Xs)
    rk, ro = _regular(sg, spec, si.torus(0.6, 0.2), *Xs)
    assert torch.equal(k.cpu(), rk) and torch.equal(o.cpu(), ro)
    with pytest.raises(sg.SgError) as e:
        sg.morton_order_noalloc(si.GridSpec((0, 0, 0), (600000, 1, 1), 0.1), Xs[0], Xs[1], Xs[2])
    assert e.value.status == sg.SG_ERR_CAPACITY


def test_noalloc_wrapper_rejects_bad_arrays(sg):
    spec = si.GridSpec((-1.0, -1.0, -0.4), (50, 50, 20), 0.01)
    X = torch.zeros(1000, device="cuda")
    with pytest.raises(ValueError):
        sg.morton_order_noalloc(spec, X, X, X.double())
    with pytest.raises(ValueError):
        sg.morton_order_noalloc(spec, X, X, X[::2])
    with pytest.raises(ValueError):
        sg.morton_order_noalloc(spec, X, X, X, order=torch.zeros(999, dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):
        sg.morton_order_noalloc(spec, X, X, X, keys=torch.zeros(1000, dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):
        sg.morton_order_noalloc(spec, X, X, X.cpu())
    # host memory passed straight to the C entry point is refused before any launch
    h = torch.zeros(1000)
    o = torch.zeros(1000, dtype=torch.int32)
    desc = sg._desc(spec)
    st = sg.lib().sg_morton_order_noalloc(C.byref(desc), 1000, *[C.c_void_p(t.data_ptr()) for t in (h, h, h)],
                                          None, C.c_void_p(o.data_ptr()),
                                          C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == sg.SG_ERR_INVALID


def test_noalloc_records_into_a_graph(sg):
    """A call recorded in a CUDA graph in global capture mode (where an
    allocation or a synchronisation by the library would end the capture
    with an error) and replayed gives the regular entry point's result."""
    shape = si.torus(0.6, 0.2)
    spec = si.GridSpec((-1.0, -1.0, -0.4), (50, 50, 20), 0.01)
    x, y, z = si.box_particles(50_000, spec.lo, spec.hi(), seed=34)
    X, Y, Z = (torch.from_numpy(v).cuda() for v in (x, y, z))
    _noalloc_raw(sg, spec, X, Y, Z)  # the device's first call loads the scratch array
    n = X.numel()
    keys = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    order = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    desc = sg._desc(spec)
    args = [C.c_void_p(t.data_ptr()) for t in (X, Y, Z, keys, order)]
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, capture_error_mode="global"):
        st = sg.lib().sg_morton_order_noalloc(C.byref(desc), n, *args,
                                              C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == sg.SG_OK
    graph.replay()
    torch.cuda.synchronize()
    rk, ro = _regular(sg, spec, shape, X, Y, Z)
    assert torch.equal(keys.cpu(), rk) and torch.equal(order.cpu(), ro)
