"""Writes the stored expected values under tests/golden/ from the oracle alone.

Run from the repository root: ``python tests/golden/make_golden.py``.  Each file
holds one value per line (repr of a float64) after a header naming what it is;
the paper prints no worked example with numbers to store (its Table 1 needs the
Congress data, which this container does not have), so these fixtures are the
oracle's own values, kept to catch unintended changes to it.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import dense  # noqa: E402
from oracle import cg as ocg  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def write(name, header, values):
    with open(os.path.join(HERE, name), "w") as f:
        for line in header:
            f.write("# " + line + "\n")
        for v in values:
            f.write(repr(float(v)) + "\n")


def main():
    wl = synth.workload_ba_small()
    g = wl.graph
    X, Y = wl.pairs(0, 16)
    write("ba_small_d2.txt",
          ["GE distance d^2 = (x - y)^T L^+ (x - y) (Section 3.1, GE equation) of the 16 pairs",
           "of the BA workload (n = 2,000, m = 3, unit weights, 10%-support pairs),",
           "oracle/dense.py eigendecomposition route (exactly c zero eigenvalues dropped)."],
          dense.ge_d2_eig(g.n, g.rowptr, g.colidx, g.w, X, Y))
    wl = synth.workload_er_large()
    g = wl.graph
    X, Y = wl.pairs(0, 2)
    d2, it, _ = ocg.ge_d2_cg(g.n, g.rowptr, g.colidx, g.w, X, Y, rtol=1e-13)
    assert np.all(it > 0)
    write("er_large_d2_first2.txt",
          ["GE distance d^2 (Section 3.1) of the first 2 pairs of the ER workload (n = 10^6",
           "generated, largest component, mean degree 10, U[0.5, 2) FP64 weights, 1%-support",
           "pairs), oracle/pcg.c FP64 Jacobi-PCG to relative residual 1e-13."],
          d2)


if __name__ == "__main__":
    main()
