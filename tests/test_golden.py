"""The stored expected values under tests/golden/ (written by make_golden.py from
the oracle alone) are reproduced by the oracle as it stands: a change to the
oracle's arithmetic shows up here."""
import os

import numpy as np
import pytest

import synth
from oracle import cg as ocg
from oracle import dense

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return np.array([float(s) for s in f if s.strip() and not s.startswith("#")])


def test_ba_small_d2():
    want = load("ba_small_d2.txt")
    wl = synth.workload_ba_small()
    g = wl.graph
    X, Y = wl.pairs(0, 16)
    got = dense.ge_d2_eig(g.n, g.rowptr, g.colidx, g.w, X, Y)
    assert want.shape == (16,)
    assert np.max(np.abs(got - want) / want) < 1e-12
    # the independent grounded-Cholesky route gives the same numbers
    got2 = dense.ge_d2_grounded(g.n, g.rowptr, g.colidx, g.w, X, Y)
    assert np.max(np.abs(got2 - want) / want) < 1e-11


@pytest.mark.slow
def test_er_large_first_pairs_d2():
    want = load("er_large_d2_first2.txt")
    wl = synth.workload_er_large()
    g = wl.graph
    X, Y = wl.pairs(0, 2)
    got, it, _ = ocg.ge_d2_cg(g.n, g.rowptr, g.colidx, g.w, X, Y, rtol=1e-13)
    assert np.all(it > 0)
    assert np.max(np.abs(got - want) / want) < 1e-11
