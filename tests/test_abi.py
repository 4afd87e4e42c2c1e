"""The C-ABI library loads without a GPU and exports every declared symbol;
the ctypes structs of the binding match the header's layout."""
import ctypes as C
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libsg():
    from paper_2512_11473_b300 import build
    build.build()
    return C.CDLL(os.path.join(ROOT, "paper_2512_11473_b300", "libsg.so"))


def test_header_declares_the_boundary():
    import paper_2512_11473_b300 as sg
    names = set(sg.declared_symbols())
    for must in ("sg_create", "sg_destroy", "sg_tag_allocate", "sg_init_sdf", "sg_gradient", "sg_reinit",
                 "sg_kernel_integrals", "sg_probe", "sg_get_field", "sg_status_sync", "sg_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(libsg):
    import paper_2512_11473_b300 as sg
    names = sg.declared_symbols()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2512_11473_b300", "libsg.so")],
                         capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    for n in names:
        assert n in exported, n
        assert hasattr(libsg, n)
    # nothing beyond the header leaks out
    assert {e for e in exported if e.startswith("sg_")} == set(names)


def test_version_callable_without_gpu(libsg):
    libsg.sg_version.restype = C.c_char_p
    assert b"sm_103a" in libsg.sg_version()


def test_struct_layout_matches_header():
    import paper_2512_11473_b300 as sg
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "sg.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(sg_shape), offsetof(sg_shape, centre), offsetof(sg_shape, rot), offsetof(sg_shape, p));
  printf("%zu %zu %zu %zu\n", sizeof(sg_grid_desc), offsetof(sg_grid_desc, dims), offsetof(sg_grid_desc, h), offsetof(sg_grid_desc, far_value));
  printf("%zu %zu %zu\n", sizeof(sg_allocator), offsetof(sg_allocator, free), offsetof(sg_allocator, ctx));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", exe, c])
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    a = [int(v) for v in lines[0].split()]
    b = [int(v) for v in lines[1].split()]
    e = [int(v) for v in lines[2].split()]
    assert a == [C.sizeof(sg.sg_shape), sg.sg_shape.centre.offset, sg.sg_shape.rot.offset, sg.sg_shape.p.offset]
    assert b == [C.sizeof(sg.sg_grid_desc), sg.sg_grid_desc.dims.offset, sg.sg_grid_desc.h.offset,
                 sg.sg_grid_desc.far_value.offset]
    assert e == [C.sizeof(sg.sg_allocator), sg.sg_allocator.free.offset, sg.sg_allocator.ctx.offset]


def test_null_arguments_rejected_without_gpu(libsg):
    """Argument checks run before any CUDA call."""
    libsg.sg_create.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    assert libsg.sg_create(None, None, None, None) == 1  # SG_ERR_INVALID
    libsg.sg_gradient.argtypes = [C.c_void_p]
    assert libsg.sg_gradient(None) == 1
    libsg.sg_destroy.argtypes = [C.c_void_p]
    assert libsg.sg_destroy(None) == 1
    # the cached autotuner and its key need a batch and a plan
    libsg.sg_batch_autotune_cached.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_char_p, C.c_void_p]
    assert libsg.sg_batch_autotune_cached(None, None, 1, b"x", None) == 1
    libsg.sg_batch_autotune_key.argtypes = [C.c_void_p, C.c_void_p, C.c_char_p, C.c_int32]
    assert libsg.sg_batch_autotune_key(None, None, C.create_string_buffer(8), 8) == 1
    libsg.sg_autotune_cache_lookup.argtypes = [C.c_char_p, C.c_char_p, C.c_void_p, C.c_void_p, C.c_void_p]
    assert libsg.sg_autotune_cache_lookup(None, b"k", None, None, None) == 1
    libsg.sg_autotune_cache_store.argtypes = [C.c_char_p, C.c_char_p, C.c_int32, C.c_int32]
    assert libsg.sg_autotune_cache_store(b"x", None, 4, 1) == 1


def test_product_refuses_to_run_without_cuda(monkeypatch):
    import torch
    import paper_2512_11473_b300 as sg
    import sg_inputs as si
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        sg.Grid(si.sphere_small()[1])


def test_product_does_not_import_oracle():
    """The product package never imports the oracle."""
    out = subprocess.run([sys.executable, "-c", "import sys, paper_2512_11473_b300; print('oracle' in sys.modules)"],
                         capture_output=True, text=True, cwd=ROOT, check=True).stdout.strip()
    assert out == "False"
    for root, _, files in os.walk(os.path.join(ROOT, "paper_2512_11473_b300")):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(root, f)).read()
                assert "import oracle" not in text and "from oracle" not in text and "sg_oracle" not in text, f
