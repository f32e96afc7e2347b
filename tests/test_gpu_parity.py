"""Parity of the CUDA path (through the C ABI) with the oracle.

Tolerances (relative error of d^2 against the FP64 oracle):
  FP64 mode  1e-6 required by the target, asserted at 1e-8 at rtol 1e-10-1e-12
             (PCG error in d^2 is the squared energy-norm error, far below rtol);
  MIXED mode 1e-8 (refined to d2_rtol 1e-10);
  FP32 mode  1e-4 (unrefined FP32 vectors).
"""
import numpy as np
import pytest

import synth
from oracle import cg as ocg
from oracle import dense

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def nvd():
    import paper_2310_11222_gb300 as m
    m.load_library()
    return m


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


def weighted(g, seed, lo=0.5, hi=2.0, dtype=np.float64):
    rng = np.random.default_rng(seed)
    return synth.csr_from_edges(g.n, g.eu, g.ev, rng.uniform(lo, hi, size=g.m).astype(dtype))


def on(x, dtype=torch.float64):
    return torch.as_tensor(x, dtype=dtype, device=DEV)


@pytest.fixture(scope="module")
def ba_small():
    wl = synth.workload_ba_small()
    X, Y = wl.pairs(0, 16)
    want = dense.ge_d2_eig(wl.graph.n, wl.graph.rowptr, wl.graph.colidx, wl.graph.w, X, Y)
    return wl.graph, X, Y, want


@pytest.mark.parametrize("fold", [False, True])
@pytest.mark.parametrize("single", [False, True])
def test_ba_small_fp64(nvd, ba_small, single, fold):
    g, X, Y, want = ba_small
    G = nvd.Graph.from_csr(g)
    d2, st = nvd.ge_distance(G, on(X), on(Y), rtol=1e-10, single_rhs=single, return_stats=True,
                             fold_direction=fold)
    assert rel(d2.cpu().numpy(), want) < 1e-8
    assert all(s["status"] == 0 and s["rel_resid"] <= 1e-10 for s in st)
    # the same iteration count either way (the same CG in exact arithmetic)
    it = [s["iters"] for s in st]
    d2c, stc = nvd.ge_distance(G, on(X), on(Y), rtol=1e-10, single_rhs=single, return_stats=True,
                               fold_direction=not fold)
    assert all(abs(a - s["iters"]) <= 1 for a, s in zip(it, stc))


def test_ba_small_against_stored_values(nvd, ba_small):
    """The stored oracle values of tests/golden/ba_small_d2.txt (make_golden.py)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ba_small_d2.txt")
    with open(path) as f:
        stored = np.array([float(v) for v in f if v.strip() and not v.startswith("#")])
    g, X, Y, _ = ba_small
    G = nvd.Graph.from_csr(g)
    d2 = nvd.ge_distance(G, on(X), on(Y), rtol=1e-10)
    assert rel(d2.cpu().numpy(), stored) < 1e-8


@pytest.mark.parametrize("kt", [1, 4, 8, 16, 32])
def test_fp64_every_tile_width(nvd, ba_small, kt):
    g, X, Y, want = ba_small
    G = nvd.Graph.from_csr(g)
    d2 = nvd.ge_distance(G, on(X[:13]), on(Y[:13]), rtol=1e-11, kt=kt)  # ragged last tile
    assert rel(d2.cpu().numpy(), want[:13]) < 1e-8


def test_ba_small_fp32(nvd, ba_small):
    g, X, Y, want = ba_small
    G = nvd.Graph.from_csr(g)
    d2 = nvd.ge_distance(G, on(X), on(Y), mode=nvd.MODE_FP32, rtol=1e-5)
    assert rel(d2.cpu().numpy(), want) < 1e-4


def test_ba_small_mixed(nvd, ba_small):
    g, X, Y, want = ba_small
    G = nvd.Graph.from_csr(g)
    d2, st = nvd.ge_distance(G, on(X), on(Y), mode=nvd.MODE_MIXED, rtol=1e-4, d2_rtol=1e-10,
                             return_stats=True)
    assert rel(d2.cpu().numpy(), want) < 1e-8
    assert all(s["status"] == 0 and s["refine_steps"] >= 2 for s in st)


def test_weighted_fp32_weights_fp64_mode(nvd):
    wl = synth.workload_ba_small(0.5)
    g = weighted(wl.graph, 3, dtype=np.float32)
    X, Y = wl.pairs(0, 8)
    want = dense.ge_d2_eig(g.n, g.rowptr, g.colidx, g.w.astype(np.float64), X, Y)
    G = nvd.Graph.from_csr(g)
    for mode, tol in [(nvd.MODE_FP64, 1e-8), (nvd.MODE_MIXED, 1e-8), (nvd.MODE_FP32, 1e-4)]:
        d2 = nvd.ge_distance(G, on(X), on(Y), mode=mode, rtol=1e-11 if mode == 0 else None,
                             d2_rtol=1e-10)
        assert rel(d2.cpu().numpy(), want) < tol, mode


def test_closed_forms_on_gpu(nvd):
    # unit path: R(0, n-1) = n - 1 (condition number ~ n^2)
    n = 400
    p = synth.csr_from_edges(n, *synth.path_graph(n), np.ones(n - 1))
    G = nvd.Graph.from_csr(p)
    x = np.zeros((2, n)); y = np.zeros((2, n))
    x[0, 0] = 1; y[0, n - 1] = 1
    x[1, 10] = 1; y[1, 110] = 1
    d2 = nvd.ge_distance(G, on(x), on(y), rtol=1e-12).cpu().numpy()
    assert rel(d2, [n - 1, 100]) < 1e-9
    # complete graph: 2 / n
    eu, ev = synth.complete_graph(30)
    K = nvd.Graph.from_csr(synth.csr_from_edges(30, eu, ev, np.full(len(eu), 2.0)))
    x = np.zeros(30); y = np.zeros(30); x[3] = 1; y[17] = 1
    assert abs(float(nvd.ge_distance(K, on(x), on(y))) - 2.0 / (30 * 2.0)) < 1e-12
    # cycle: h (n - h) / n
    C = nvd.Graph.from_csr(synth.csr_from_edges(50, *synth.cycle_graph(50), np.ones(50)))
    x = np.zeros(50); y = np.zeros(50); x[0] = 1; y[20] = 1
    assert abs(float(nvd.ge_distance(C, on(x), on(y), rtol=1e-12)) - 20 * 30 / 50) < 1e-9


def test_disconnected_interleaved_components_and_isolated_nodes(nvd):
    """Components that are not contiguous node ranges (internal relabelling), isolated
    nodes (singletons) and z_out in the user's node order."""
    rng = np.random.default_rng(5)
    parts = []
    for seed, n in [(1, 40), (2, 25), (3, 1), (4, 30), (5, 1)]:
        r = np.random.default_rng(seed)
        if n == 1:
            parts.append(synth.csr_from_edges(1, np.empty(0, np.int64), np.empty(0, np.int64), np.empty(0)))
        else:
            eu, ev = synth.barabasi_albert(n, 2, r)
            parts.append(synth.csr_from_edges(n, eu, ev, r.uniform(0.5, 2, size=len(eu))))
    gu, _ = synth.disjoint_union(parts)
    perm = rng.permutation(gu.n)            # interleave the components
    g = synth.csr_from_edges(gu.n, perm[gu.eu], perm[gu.ev], gu.ew)
    X, Y = rng.random((6, g.n)), rng.random((6, g.n))
    want = dense.ge_d2_eig(g.n, g.rowptr, g.colidx, g.w, X, Y)
    Zw = dense.ge_z_dense(g.n, g.rowptr, g.colidx, g.w, X, Y)
    G = nvd.Graph.from_csr(g)
    assert G.info()["ncomp"] == 5
    for mode, tol in [(0, 1e-8), (2, 1e-8), (1, 1e-4)]:
        d2, z = nvd.ge_distance(G, on(X), on(Y), mode=mode, rtol=1e-11 if mode == 0 else None,
                                d2_rtol=1e-10, return_z=True)
        assert rel(d2.cpu().numpy(), want) < tol
        zt = z.cpu().numpy()
        assert np.max(np.abs(zt - Zw)) < tol * 10 * np.max(np.abs(Zw))


def test_heavy_rows_split_over_ctas(nvd):
    """A hub of degree 5000 (> every sub-item budget) forces the split-row path."""
    rng = np.random.default_rng(7)
    n = 6000
    eu = np.concatenate([np.zeros(5000, np.int64), rng.integers(1, n, 4000)])
    ev = np.concatenate([np.arange(1, 5001), rng.integers(1, n, 4000)])
    eu, ev = synth.graphs._canonical_unique(eu, ev, n)
    nn, eu, ev, _ = synth.largest_component(n, eu, ev)
    g = synth.csr_from_edges(nn, eu, ev, rng.uniform(0.5, 2, size=len(eu)))
    assert np.diff(g.rowptr).max() >= 5000
    X, Y = rng.random((5, g.n)), rng.random((5, g.n))
    want = ocg.ge_d2_cg(g.n, g.rowptr, g.colidx, g.w, X, Y, rtol=1e-13)[0]
    G = nvd.Graph.from_csr(g)
    for kt in (1, 4, 8, 16, 32):
        d2 = nvd.ge_distance(G, on(X), on(Y), rtol=1e-12, kt=kt)
        assert rel(d2.cpu().numpy(), want) < 1e-8, kt
    d2 = nvd.ge_distance(G, on(X), on(Y), mode=nvd.MODE_MIXED, d2_rtol=1e-10)
    assert rel(d2.cpu().numpy(), want) < 1e-8


def test_laplacian_apply_matches_definition(nvd):
    wl = synth.workload_grad(0.002)
    g = wl.graph
    rng = np.random.default_rng(1)
    X = rng.standard_normal((3, g.n))
    L = dense.laplacian_dense(g.n, g.rowptr, g.colidx, g.w.astype(np.float64)) if g.n <= 3000 else None
    G = nvd.Graph.from_csr(g)
    y = nvd.laplacian_apply(G, on(X)).cpu().numpy()
    want = X @ L
    assert np.max(np.abs(y - want)) < 1e-10 * np.max(np.abs(want))
    y32 = nvd.laplacian_apply(G, on(X, torch.float32)).cpu().numpy()
    assert np.max(np.abs(y32 - want)) < 1e-5 * np.max(np.abs(want))


def test_host_inputs_path_matches_device_path(nvd, ba_small):
    g, X, Y, want = ba_small
    G = nvd.Graph.from_csr(g)
    a = nvd.ge_distance(G, on(X), on(Y), rtol=1e-10).cpu().numpy()
    b = nvd.ge_distance(G, torch.from_numpy(X), torch.from_numpy(Y), rtol=1e-10).numpy()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("mode,kw", [(0, dict(single_rhs=True)), (0, dict(kt=4)), (2, dict(kt=4))])
def test_host_inputs_many_tiles_with_z(nvd, mode, kw):
    """Host inputs over 5+ tiles (the two staging slots are each reused) with z_out on a
    graph with interleaved components and an isolated node (node permutation): d^2 and
    z equal the device-input path bitwise, stats per pair included."""
    rng = np.random.default_rng(21)
    parts = []
    for seed, n in [(1, 400), (2, 1), (3, 250)]:
        r = np.random.default_rng(seed)
        if n == 1:
            parts.append(synth.csr_from_edges(1, np.empty(0, np.int64), np.empty(0, np.int64), np.empty(0)))
        else:
            eu, ev = synth.barabasi_albert(n, 3, r)
            parts.append(synth.csr_from_edges(n, eu, ev, r.uniform(0.5, 2, size=len(eu))))
    gu, _ = synth.disjoint_union(parts)
    perm = rng.permutation(gu.n)
    g = synth.csr_from_edges(gu.n, perm[gu.eu], perm[gu.ev], gu.ew)
    X, Y = rng.random((18, g.n)), rng.random((18, g.n))
    G = nvd.Graph.from_csr(g)
    a, za, sa = nvd.ge_distance(G, on(X), on(Y), mode=mode, rtol=1e-10, return_z=True, return_stats=True, **kw)
    b, zb, sb = nvd.ge_distance(G, torch.from_numpy(X), torch.from_numpy(Y), mode=mode, rtol=1e-10,
                                return_z=True, return_stats=True, **kw)
    assert np.array_equal(a.cpu().numpy(), b.numpy())
    assert np.array_equal(za.cpu().numpy(), zb.numpy())
    assert [s["iters"] for s in sa] == [s["iters"] for s in sb]
    want = dense.ge_d2_eig(g.n, g.rowptr, g.colidx, g.w, X, Y)
    assert rel(b.numpy(), want) < 1e-8


def test_repeatable_bitwise(nvd, ba_small):
    g, X, Y, _ = ba_small
    G = nvd.Graph.from_csr(g)
    a = nvd.ge_distance(G, on(X), on(Y), mode=nvd.MODE_MIXED).cpu().numpy()
    b = nvd.ge_distance(G, on(X), on(Y), mode=nvd.MODE_MIXED).cpu().numpy()
    assert np.array_equal(a, b)


def test_input_validation_and_cleaning(nvd):
    base = weighted(synth.workload_ba_small(0.05).graph, 9)
    n = base.n
    rng = np.random.default_rng(2)
    X, Y = rng.random((2, n)), rng.random((2, n))
    want = dense.ge_d2_eig(n, base.rowptr, base.colidx, base.w, X, Y)
    # asymmetric weights
    w = base.w.copy(); w[0] *= 1.5
    with pytest.raises(nvd.NvdError) as e:
        nvd.Graph(base.rowptr, base.colidx, w)
    assert e.value.status == 2
    # non-positive / NaN weight
    for bad in (0.0, -1.0, np.nan, np.inf):
        w = base.w.copy(); w[3] = bad
        with pytest.raises(nvd.NvdError) as e:
            nvd.Graph(base.rowptr, base.colidx, w)
        assert e.value.status == 3
    # column out of range / bad rowptr
    c = base.colidx.copy(); c[0] = n + 5
    with pytest.raises(nvd.NvdError) as e:
        nvd.Graph(base.rowptr, c, base.w)
    assert e.value.status == 1
    rp = base.rowptr.copy(); rp[-1] += 1
    with pytest.raises(nvd.NvdError):
        nvd.Graph(rp, base.colidx, base.w)
    # unsorted rows, split duplicates and a self-loop are cleaned, result unchanged
    rows = np.repeat(np.arange(n), np.diff(base.rowptr))
    r2 = np.concatenate([rows, rows, [4]])
    c2 = np.concatenate([base.colidx, base.colidx, [4]])
    w2 = np.concatenate([0.25 * base.w, 0.75 * base.w, [3.0]])
    order = np.lexsort((-c2, r2))           # columns descending within each row
    r2, c2, w2 = r2[order], c2[order], w2[order]
    rp2 = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(r2, minlength=n), out=rp2[1:])
    G = nvd.Graph(rp2, c2.astype(np.int32), w2)
    assert G.info()["nnz"] == base.nnz
    d2 = nvd.ge_distance(G, on(X), on(Y), rtol=1e-12).cpu().numpy()
    assert rel(d2, want) < 1e-9
    # gradient on the cleaned graph lands on the user's entries (self-loop gets 0)
    _, z = nvd.ge_distance(G, on(X), on(Y), rtol=1e-12, return_z=True)
    gw, _, _ = nvd.ge_grad(G, z, torch.ones(2, dtype=torch.float64, device=DEV))
    gw = gw.cpu().numpy()
    gref, _, _ = dense.ge_grad_dense(n, base.rowptr, base.colidx, base.w, X, Y, np.ones(2))
    # each duplicate entry carries the full per-entry derivative of its merged entry
    key_ref = {(int(a), int(b)): v for a, b, v in zip(rows, base.colidx, gref)}
    for e in range(len(r2)):
        if r2[e] == c2[e]:
            assert gw[e] == 0.0
        else:
            assert abs(gw[e] - key_ref[(int(r2[e]), int(c2[e]))]) <= 1e-8 * np.max(np.abs(gref))


def test_gradients_match_dense_oracle(nvd):
    wl = synth.workload_grad(0.0006)        # BA m = 5, lognormal(0, 0.5) FP32 weights, n = 600
    g = wl.graph
    X, Y = wl.pairs(0, 6)
    gbar = np.linspace(0.5, 1.5, 6)
    w64 = g.w.astype(np.float64)
    gw_ref, gx_ref, gy_ref = dense.ge_grad_dense(g.n, g.rowptr, g.colidx, w64, X, Y, gbar)
    G = nvd.Graph.from_csr(g)
    for mode in (nvd.MODE_FP64, nvd.MODE_MIXED):
        d2, z = nvd.ge_distance(G, on(X), on(Y), mode=mode, rtol=1e-12 if mode == 0 else None,
                                d2_rtol=1e-12, return_z=True)
        gw, gx, gy = nvd.ge_grad(G, z, on(gbar))
        assert gw.dtype == torch.float32
        assert np.max(np.abs(gw.cpu().numpy() - gw_ref)) <= 1e-5 * np.max(np.abs(gw_ref))
        assert np.max(np.abs(gx.cpu().numpy() - gx_ref)) <= 1e-8 * np.max(np.abs(gx_ref))
        assert np.max(np.abs(gy.cpu().numpy() + gx_ref)) <= 1e-8 * np.max(np.abs(gx_ref))


def test_autograd_function(nvd):
    wl = synth.workload_grad(0.0004)
    g = wl.graph
    X, Y = wl.pairs(0, 3)
    G = nvd.Graph.from_csr(g)
    x = on(X, torch.float32).requires_grad_()
    y = on(Y, torch.float32).requires_grad_()
    w = torch.as_tensor(g.w, device=DEV).requires_grad_()
    d2 = nvd.ge_distance_autograd(G, x, y, w, mode=nvd.MODE_MIXED)
    (d2 * torch.tensor([1.0, 2.0, 3.0], dtype=torch.float64, device=DEV)).sum().backward()
    gw_ref, gx_ref, _ = dense.ge_grad_dense(g.n, g.rowptr, g.colidx, g.w.astype(np.float64),
                                             X.astype(np.float32).astype(np.float64),
                                             Y.astype(np.float32).astype(np.float64), [1.0, 2.0, 3.0])
    assert np.max(np.abs(w.grad.cpu().numpy() - gw_ref)) <= 1e-4 * np.max(np.abs(gw_ref))
    assert np.max(np.abs(x.grad.cpu().numpy() - gx_ref)) <= 1e-5 * np.max(np.abs(gx_ref))
    assert np.max(np.abs(y.grad.cpu().numpy() + gx_ref)) <= 1e-5 * np.max(np.abs(gx_ref))


@pytest.fixture(scope="module")
def d2stop_cases():
    """Graphs of the four synthetic families at n = 20,000 (ER mean degree 8, BA m = 4,
    WS k = 4, SBM mean degree 8, U[0.5, 2) weights) and the BA workload graph, each
    with 6 pairs of 10% support and 2 indicator pairs, and the oracle's d^2 (C FP64
    CG at relative residual 1e-13)."""
    out = []
    for model, kdeg in [("er", 8), ("ba", 8), ("ws", 4), ("sbm", 8)]:
        g0 = synth.sweep_graph(model, 20000, kdeg, seed=40 + kdeg)
        out.append(weighted(g0, 41))
    out.append(synth.workload_ba_small().graph)
    cases = []
    for g in out:
        X, Y = synth.sparse_uniform_pairs(g.n, 6, 0.10, 77)
        lab, _ = ocg.components(g.n, g.rowptr, g.colidx)
        big = np.nonzero(lab == np.argmax(np.bincount(lab)))[0]
        rng = np.random.default_rng(g.n)
        Xi, Yi = np.zeros((2, g.n)), np.zeros((2, g.n))
        for j in range(2):
            a, b = rng.choice(big, 2, replace=False)
            Xi[j, a] = 1.0
            Yi[j, b] = 1.0
        X, Y = np.vstack([X, Xi]), np.vstack([Y, Yi])
        want, it, _ = ocg.ge_d2_cg(g.n, g.rowptr, g.colidx, g.w.astype(np.float64), X, Y, rtol=1e-13)
        assert np.all(it > 0)
        cases.append((g, X, Y, want))
    return cases


@pytest.mark.parametrize("kw", [dict(single_rhs=True), dict(single_rhs=True, persistent=True),
                                dict(single_rhs=True, fold_direction=True), dict(kt=8),
                                dict(kt=8, persistent=True, fold_direction=True)])
def test_d2_stop_meets_its_tolerance(nvd, d2stop_cases, kw):
    """NVD_SOLVE_D2_STOP: every pair's d^2 within d2_rtol of the oracle (1e-6 and 1e-8),
    with fewer iterations than the residual test at rtol 1e-10 needs."""
    for g, X, Y, want in d2stop_cases:
        G = nvd.Graph.from_csr(g)
        _, st_ref = nvd.ge_distance(G, on(X), on(Y), rtol=1e-10, return_stats=True, **kw)
        for tol in (1e-6, 1e-8):
            d2, st = nvd.ge_distance(G, on(X), on(Y), rtol=1e-14, d2_stop=True, d2_rtol=tol,
                                     return_stats=True, **kw)
            assert all(s["status"] == 0 for s in st)
            assert rel(d2.cpu().numpy(), want) <= tol, (g.n, tol)
            assert sum(s["iters"] for s in st) < sum(s["iters"] for s in st_ref)


def test_d2_stop_fp32_and_invalid_uses(nvd, d2stop_cases):
    g, X, Y, want = d2stop_cases[0]
    G = nvd.Graph.from_csr(g)
    d2 = nvd.ge_distance(G, on(X), on(Y), mode=nvd.MODE_FP32, rtol=1e-6, d2_stop=True, d2_rtol=1e-4, kt=8)
    assert rel(d2.cpu().numpy(), want) <= 1e-4
    for bad in (dict(mode=nvd.MODE_MIXED, d2_stop=True), dict(d2_stop=True, d2_rtol=1.0)):
        with pytest.raises(nvd.NvdError) as e:
            nvd.ge_distance(G, on(X), on(Y), **bad)
        assert e.value.status == 1


@pytest.mark.slow
def test_er_large_full_size_single_rhs(nvd):
    """ER n = 1e6 (largest component), mean degree 10, FP64 weights, 8 pairs solved one
    right-hand side at a time in FP64 -- the workload the bench times -- against the
    C FP64 CG oracle at relative residual 1e-12."""
    wl = synth.workload_er_large()
    g = wl.graph
    X, Y = wl.pairs(0, 8)
    want, it, rr = ocg.ge_d2_cg(g.n, g.rowptr, g.colidx, g.w, X, Y, rtol=1e-12)
    assert np.all(it > 0)
    G = nvd.Graph.from_csr(g)
    d2, st = nvd.ge_distance(G, on(X), on(Y), rtol=1e-10, single_rhs=True, return_stats=True)
    assert rel(d2.cpu().numpy(), want) < 1e-8
    assert all(s["status"] == 0 for s in st)
    d2b = nvd.ge_distance(G, on(X), on(Y), rtol=1e-10)          # batched RHS, same answer
    assert rel(d2b.cpu().numpy(), want) < 1e-8
    # the accuracy the metric asks (d^2 within 1e-6) by the d^2 stop, in far fewer iterations
    d2s, sts = nvd.ge_distance(G, on(X), on(Y), rtol=1e-14, single_rhs=True, d2_stop=True, d2_rtol=1e-6,
                               return_stats=True)
    assert rel(d2s.cpu().numpy(), want) <= 1e-6
    assert max(s["iters"] for s in sts) < min(s["iters"] for s in st)
