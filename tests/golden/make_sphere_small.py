"""Write tests/golden/sphere_small_oracle.txt from the oracle alone.

The file is a regression record of the oracle, not a pin of it: it holds
what the FP64 oracle computes for the small sphere (unit sphere, h = 0.05;
tagging, tables, initialisation, gradient, 20 reinit sweeps at CFL 0.5,
exact kernel integrals), so that any later change of the oracle's arithmetic
shows up in tests/test_golden.py and has to be justified by the passage of
the paper it follows.  The pins of the oracle against the mathematics are in
tests/test_oracle_pins.py.

Usage: python tests/golden/make_sphere_small.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import sg_inputs as si  # noqa: E402

OUT = os.path.join(HERE, "sphere_small_oracle.txt")
POINTS = (0, 21, 42, 63)  # data points d = i + 4 j + 16 k of each sampled package


def compute():
    """The oracle pipeline on the small sphere: counts and sampled values."""
    shape, spec = si.sphere_small()
    cell_pkg, cell_type, P, ties = oracle.tag(spec, shape)
    pkg_cell, pkg_type, nbr = oracle.tables(spec, cell_pkg, cell_type, P)
    phi0 = oracle.init_sdf(spec, shape, P, pkg_cell)
    g = oracle.gradient(spec, nbr, phi0)
    phi = oracle.reinit(spec, nbr, phi0, 20, 0.5)
    w = oracle.kernel_integrals(spec, nbr, phi)
    counts = {"P": P, "core": int((pkg_type == 2).sum()), "inner": int((pkg_type == 3).sum()), "ties": ties}
    pkgs = np.linspace(2, P - 1, 16).round().astype(int)
    fields = {"phi0": phi0, "gx": g[0], "gy": g[1], "gz": g[2], "phi20": phi, "W": w[0], "Gx": w[1], "Gy": w[2],
              "Gz": w[3]}
    rows = []
    for p in pkgs:
        for d in POINTS:
            rows.append((int(p), d) + tuple(float(fields[k][p, d]) for k in fields))
    sums = {k: float(np.abs(v[2:]).sum()) for k, v in fields.items()}
    return counts, list(fields), rows, sums


def main():
    counts, names, rows, sums = compute()
    with open(OUT, "w") as f:
        f.write("# Regression record of the FP64 oracle on the small sphere (unit sphere at\n")
        f.write("# the origin, [-1.5, 1.5]^3, h = 0.05): written by make_sphere_small.py,\n")
        f.write("# which calls only oracle/ and the input shapes of sg_inputs.  Not a pin.\n")
        for k, v in counts.items():
            f.write("count %s %d\n" % (k, v))
        for k, v in sums.items():
            f.write("abssum %s %r\n" % (k, v))
        f.write("columns package point %s\n" % " ".join(names))
        for r in rows:
            f.write("value %d %d %s\n" % (r[0], r[1], " ".join(repr(x) for x in r[2:])))
    print(OUT)


if __name__ == "__main__":
    main()
