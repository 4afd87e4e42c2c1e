"""Stored fixtures under tests/golden/.

* paper_table1.txt: values the paper prints ("Performance Evaluation",
  Table 1 and its paragraph).  The synthetic Table 1 body and the benchmark's
  context figures must be those values.
* sphere_small_oracle.txt: a regression record of the FP64 oracle on the
  small sphere, written by tests/golden/make_sphere_small.py from the oracle
  alone.  Recomputing it must give the stored numbers, so that a change of
  the oracle's arithmetic cannot pass unnoticed.
"""
import importlib.util
import os

import pytest

import sg_inputs as si

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _pairs(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_paper_table1_body_and_context():
    t = _pairs("paper_table1.txt")
    shape, spec = si.shelled_sphere()
    assert shape.kind == si.SHELL
    assert shape.centre == (t["shell_centre_x"], t["shell_centre_y"], t["shell_centre_z"])
    assert (shape.p[0], shape.p[1]) == (t["shell_inner_radius"], t["shell_outer_radius"])
    assert spec.h == t["resolution"] == 1.0 / 1024
    import bench
    for k, v in bench.PAPER_TABLE1_MS.items():
        assert v == t[k], k


def _make():
    spec = importlib.util.spec_from_file_location("make_sphere_small", os.path.join(GOLDEN, "make_sphere_small.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_sphere_small_oracle_record():
    counts, names, rows, sums = _make().compute()
    stored_counts, stored_sums, stored_rows, cols = {}, {}, [], None
    for line in open(os.path.join(GOLDEN, "sphere_small_oracle.txt")):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "count":
            stored_counts[f[1]] = int(f[2])
        elif f[0] == "abssum":
            stored_sums[f[1]] = float(f[2])
        elif f[0] == "columns":
            cols = f[3:]
        elif f[0] == "value":
            stored_rows.append((int(f[1]), int(f[2])) + tuple(float(x) for x in f[3:]))
    assert counts == stored_counts
    assert cols == names
    for k, v in sums.items():
        assert v == pytest.approx(stored_sums[k], rel=1e-12), k
    assert len(rows) == len(stored_rows) == 64
    for got, want in zip(rows, stored_rows):
        assert got[:2] == want[:2]
        for a, b in zip(got[2:], want[2:]):
            assert a == pytest.approx(b, rel=1e-12, abs=1e-14), got[:2]
