"""Host-side checks of the seeded input generators (shapes, counts, structure)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import synth


def _adj(g):
    return sp.csr_matrix((g.w, g.colidx, g.rowptr), shape=(g.n, g.n))


def _check_csr(g):
    A = _adj(g)
    assert g.rowptr[0] == 0 and g.rowptr[-1] == g.colidx.shape[0]
    assert np.all(np.diff(g.rowptr) >= 0)
    assert abs(A - A.T).max() == 0
    assert A.diagonal().max(initial=0) == 0
    for u in range(0, g.n, max(1, g.n // 50)):
        row = g.colidx[g.rowptr[u]:g.rowptr[u + 1]]
        assert np.all(np.diff(row) > 0)
    assert g.nnz == 2 * g.m


def test_er_counts_and_determinism():
    rng = np.random.default_rng(0)
    eu, ev = synth.erdos_renyi_gnm(1000, 5000, rng)
    assert len(eu) == 5000 and np.all(eu < ev)
    assert len(np.unique(eu * 1000 + ev)) == 5000
    eu2, ev2 = synth.erdos_renyi_gnm(1000, 5000, np.random.default_rng(0))
    assert np.array_equal(eu, eu2) and np.array_equal(ev, ev2)


def test_ba_structure():
    eu, ev = synth.barabasi_albert(500, 3, np.random.default_rng(1))
    assert len(eu) == 3 + 3 * (500 - 4)
    deg = np.bincount(np.concatenate([eu, ev]), minlength=500)
    assert deg.min() >= 1 and deg[4:].min() >= 3
    assert deg.max() > 20            # preferential attachment grows hubs


def test_ws_structure():
    eu, ev = synth.watts_strogatz(1000, 10, 0.1, np.random.default_rng(2))
    assert len(eu) == 1000 * 5
    ring = np.abs(ev - eu)
    ring = np.minimum(ring, 1000 - ring)
    frac_rewired = np.mean(ring > 5)
    assert 0.05 < frac_rewired < 0.15


def test_powerlaw_degree_bounds():
    eu, ev = synth.configuration_model_powerlaw(20000, 2.3, 2, 1000, np.random.default_rng(3))
    deg = np.bincount(np.concatenate([eu, ev]), minlength=20000)
    assert deg.max() <= 1000
    assert np.mean(deg) > 3.0


def test_workloads_small_scale():
    for name, fn in synth.WORKLOADS.items():
        scale = 1.0 if name == "ba_small" else 0.003
        wl = fn(scale) if name != "batched" else fn(0.02, n_graphs=4)
        g = wl.graph
        _check_csr(g)
        ncomp = csg.connected_components(_adj(g))[0]
        if name == "batched":
            assert ncomp == 4
        else:
            assert ncomp == 1
        if name != "batched":
            X, Y = wl.pairs(0, 3)
            assert X.shape == (3, g.n)
            assert np.allclose(X.sum(1), 1.0) and np.allclose(Y.sum(1), 1.0)
            X1, _ = wl.pairs(1, 1)
            assert np.array_equal(X1[0], X[1])


def test_sbm():
    n, eu, ev = synth.stochastic_block_model([50, 60, 40], 0.2, 0.01, np.random.default_rng(4))
    assert n == 150 and np.all(eu < ev)
    same = (eu // 50 == ev // 50) & (eu < 100) & (ev < 100)
    assert same.sum() > 0


@pytest.mark.parametrize("model", ["er", "ba", "ws", "sbm"])
def test_sweep_graphs_match_edge_counts(model):
    """The sweep models are compared at the same number of edges, n * mean_degree / 2."""
    for n, k in [(2000, 8.0), (3000, 4.0)]:
        g = synth.sweep_graph(model, n, k, seed=1)
        assert g.n == n
        nnz = int(g.rowptr[-1])
        assert abs(nnz / n - k) <= 0.1 * k, (model, n, k, nnz / n)
        # symmetric, no self-loops, sorted rows
        rows = np.repeat(np.arange(n), np.diff(g.rowptr))
        assert np.all(rows != g.colidx)
        fwd = set(zip(rows.tolist(), g.colidx.tolist()))
        assert all((v, u) in fwd for u, v in list(fwd)[:2000])
    assert synth.sweep_graph(model, 2000, 8.0, seed=3).structure_hash() == \
        synth.sweep_graph(model, 2000, 8.0, seed=3).structure_hash()
