"""Batched solve (many graphs as one block-diagonal Laplacian: host-driven launches over
all graphs by default, or one persistent cooperative launch in a CUDA graph) and the
persistent single-graph solve, against the oracle and the host-driven path."""
import numpy as np
import pytest

import synth
from oracle import cg as ocg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def nvd():
    import paper_2310_11222_gb300 as m
    m.load_library()
    return m


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


def on(x, dtype=torch.float64):
    return torch.as_tensor(x, dtype=dtype, device=DEV)


@pytest.fixture(scope="module")
def small_batch():
    graphs = [synth.workloads.batched_graph(gi, scale=0.02) for gi in list(range(4)) + list(range(32, 36))]
    pairs = []
    for gi, g in zip(list(range(4)) + list(range(32, 36)), graphs):
        pairs.append(synth.workloads.batched_pairs(g, gi))
    want = []
    for g, (X, Y) in zip(graphs, pairs):
        d2, it, _ = ocg.ge_d2_cg(g.n, g.rowptr, g.colidx, g.w, X, Y, rtol=1e-12)
        assert np.all(it >= 0)
        want.append(d2)
    return graphs, pairs, want


@pytest.mark.parametrize("persistent", [False, True])
@pytest.mark.parametrize("mode,rtol,tol", [(0, 1e-10, 1e-8), (1, 1e-6, 1e-4)])
def test_batched_matches_oracle(nvd, small_batch, mode, rtol, tol, persistent):
    graphs, pairs, want = small_batch
    G = [nvd.Graph.from_csr(g) for g in graphs]
    xs = [on(X) for X, _ in pairs]
    ys = [on(Y) for _, Y in pairs]
    d2, st = nvd.ge_distance_batched(G, xs, ys, mode=mode, rtol=rtol, return_stats=True, persistent=persistent)
    d2 = d2.numpy()
    off = 0
    for w in want:
        assert rel(d2[off:off + len(w)], w) < tol
        off += len(w)
    assert all(s["status"] == 0 for s in st)
    # a second call (the persistent form replays its captured launch) gives the identical answer
    d2b = nvd.ge_distance_batched(G, xs, ys, mode=mode, rtol=rtol, persistent=persistent).numpy()
    assert np.array_equal(d2, d2b)


@pytest.mark.parametrize("mode,tol_p", [(0, 1e-12), (1, 1e-6)])
def test_batched_host_loop_agrees_with_persistent(nvd, small_batch, mode, tol_p):
    """The host-driven launches and the persistent kernel run the same phases over the
    union graph; their results agree to rounding, with the same iteration counts."""
    graphs, pairs, _ = small_batch
    G = [nvd.Graph.from_csr(g) for g in graphs]
    xs = [on(X) for X, _ in pairs]
    ys = [on(Y) for _, Y in pairs]
    rtol = 1e-10 if mode == 0 else 1e-6
    h, sh = nvd.ge_distance_batched(G, xs, ys, mode=mode, rtol=rtol, return_stats=True)
    p, sp_ = nvd.ge_distance_batched(G, xs, ys, mode=mode, rtol=rtol, return_stats=True, persistent=True)
    assert rel(h.numpy(), p.numpy()) < tol_p
    assert [s["iters"] for s in sh] == [s["iters"] for s in sp_]


def test_batched_equals_independent_solves(nvd, small_batch):
    graphs, pairs, _ = small_batch
    G = [nvd.Graph.from_csr(g) for g in graphs]
    xs = [on(X) for X, _ in pairs]
    ys = [on(Y) for _, Y in pairs]
    d2 = nvd.ge_distance_batched(G, xs, ys, mode=nvd.MODE_FP64, rtol=1e-10).numpy()
    off = 0
    for g, x, y in zip(G, xs, ys):
        one = nvd.ge_distance(g, x, y, rtol=1e-10, kt=16).cpu().numpy()
        assert rel(d2[off:off + len(one)], one) < 1e-9
        off += len(one)


def test_batched_uneven_pair_counts_and_multiple_tiles(nvd, small_batch):
    graphs, pairs, want = small_batch
    G = [nvd.Graph.from_csr(g) for g in graphs[:3]]
    ks = [5, 32, 17]
    xs = [on(pairs[i][0][:k]) for i, k in enumerate(ks)]
    ys = [on(pairs[i][1][:k]) for i, k in enumerate(ks)]
    d2 = nvd.ge_distance_batched(G, xs, ys, mode=nvd.MODE_FP64, rtol=1e-10).numpy()
    off = 0
    for i, k in enumerate(ks):
        assert rel(d2[off:off + k], want[i][:k]) < 1e-8
        off += k


@pytest.mark.parametrize("fold", [False, True])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("kt", [1, 8, 32])
def test_persistent_single_graph_bitwise_equals_host_loop(nvd, mode, kt, fold):
    """The persistent kernel runs the per-slice register SpMM: with that gather engine
    the host loop runs the same sums in the same order (bitwise equal); with the
    stream engine (multi-column tiles) only the grouping of the inner products
    differs."""
    wl = synth.workload_ba_small()
    g = wl.graph
    X, Y = wl.pairs(0, 12)
    G = nvd.Graph.from_csr(g)
    if mode == 0 and kt == 32:
        kt = 16
    b, zb = nvd.ge_distance(G, on(X), on(Y), mode=mode, kt=kt, persistent=True, return_z=True,
                            fold_direction=fold)
    G.set_tuning(mode=mode, gather=nvd.GATHER_SLICES)
    a, za = nvd.ge_distance(G, on(X), on(Y), mode=mode, kt=kt, return_z=True, fold_direction=fold)
    assert torch.equal(a, b)
    assert torch.equal(za, zb)
    G.set_tuning(mode=mode, gather=nvd.GATHER_STREAM)
    t, zt = nvd.ge_distance(G, on(X), on(Y), mode=mode, kt=kt, return_z=True, fold_direction=fold)
    tol = 1e-12 if mode == 0 else 1e-5
    assert rel(t.cpu().numpy(), b.cpu().numpy()) < tol


@pytest.mark.parametrize("mode,tol", [(0, 1e-11), (1, 1e-5)])
def test_batched_folded_direction_matches_three_kernel_iteration(nvd, small_batch, mode, tol):
    graphs, pairs, want = small_batch
    G = [nvd.Graph.from_csr(g) for g in graphs]
    xs = [on(X) for X, _ in pairs]
    ys = [on(Y) for _, Y in pairs]
    rtol = 1e-10 if mode == 0 else 1e-6
    for persistent in (False, True):
        a = nvd.ge_distance_batched(G, xs, ys, mode=mode, rtol=rtol, persistent=persistent).numpy()
        b = nvd.ge_distance_batched(G, xs, ys, mode=mode, rtol=rtol, fold_direction=True,
                                    persistent=persistent).numpy()
        assert rel(a, b) < tol


@pytest.fixture(scope="module")
def full_batch():
    """The 64-graph batch (node counts log-uniform in [1e3, 2e5]; 32 BA, 32 WS), 32 pairs
    each, with the FP64 oracle's d^2 of every pair (C CG at rtol 1e-12)."""
    wl = synth.workload_batched()
    X, Y = wl.pairs(0, 32)
    want = []
    for gi, g in enumerate(wl.graphs):
        d2, it, _ = ocg.ge_d2_cg(g.n, g.rowptr, g.colidx, g.w.astype(np.float64), X[gi], Y[gi], rtol=1e-12)
        assert np.all(it > 0)
        want.append(d2)
    return wl, X, Y, np.concatenate(want)


@pytest.mark.slow
@pytest.mark.parametrize("persistent", [False, True])
@pytest.mark.parametrize("mode,rtol,tol", [(1, 1e-6, 1e-4), (0, 1e-11, 1e-8)])
def test_batched_full_size_all_graphs(nvd, full_batch, mode, rtol, tol, persistent):
    """All 2,048 pairs of the full batch (the host-driven launches, or one persistent
    launch per tile) against the oracle: FP32 vectors with FP64 reductions at the
    unrefined-FP32 tolerance 1e-4, and FP64 at 1e-8."""
    wl, X, Y, want = full_batch
    G = [nvd.Graph.from_csr(g) for g in wl.graphs]
    xs = [on(x) for x in X]
    ys = [on(y) for y in Y]
    d2, st = nvd.ge_distance_batched(G, xs, ys, mode=mode, rtol=rtol, return_stats=True, persistent=persistent)
    d2 = d2.numpy()
    assert np.all(np.isfinite(d2)) and np.all(d2 > 0)
    assert all(s["status"] == 0 for s in st)
    assert rel(d2, want) < tol


@pytest.mark.slow
@pytest.mark.parametrize("mode,rtol,tol", [(1, 1e-6, 1e-4), (0, 1e-12, 1e-9)])
def test_batched_more_owner_columns_than_the_grid_has_threads(nvd, mode, rtol, tol):
    """3,000 small random graphs (6..23 nodes, some disconnected) with 32 pairs each:
    96,000 (graph, pair) columns, more than one co-resident wave of the persistent
    kernel has threads, so the per-column results are collected in grid-stride
    loops; every d^2 against the dense oracle."""
    from oracle import dense
    rng = np.random.default_rng(77)
    graphs, xs, ys, want = [], [], [], []
    for _ in range(3000):
        n = int(rng.integers(6, 24))
        eu, ev = synth.random_gnp_small(n, 0.35, rng)
        if len(eu) == 0:
            eu, ev = np.array([0]), np.array([1])
        g = synth.csr_from_edges(n, eu, ev, rng.uniform(0.5, 2.0, len(eu)))
        X, Y = rng.random((32, n)), rng.random((32, n))
        graphs.append(g)
        xs.append(X)
        ys.append(Y)
        want.append(dense.ge_d2_eig(g.n, g.rowptr, g.colidx, g.w, X, Y))
    want = np.concatenate(want)
    G = [nvd.Graph.from_csr(g) for g in graphs]
    for persistent in (True, False):
        d2 = nvd.ge_distance_batched(G, [on(x) for x in xs], [on(y) for y in ys], mode=mode, rtol=rtol,
                                     persistent=persistent).numpy()
        pos = want > 1e-12
        assert rel(d2[pos], want[pos]) < tol
        assert np.all(np.abs(d2[~pos]) < 1e-9)
