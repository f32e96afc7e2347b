"""The autotuner (nvd_graph_tune) and explicit settings (nvd_graph_set_tuning): every
work decomposition it can pick gives the oracle's d^2, and the tuned setting is the
one later calls use."""
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
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


def on(x):
    return torch.as_tensor(x, dtype=torch.float64, device=DEV)


@pytest.fixture(scope="module")
def hub_graph():
    """BA-like graph plus a hub of degree 3000 and a few rows around every light-row limit."""
    rng = np.random.default_rng(11)
    n = 5000
    eu, ev = synth.barabasi_albert(n, 3, rng)
    extra_u = [np.zeros(3000, np.int64)]
    extra_v = [np.arange(1, 3001)]
    for hub, deg in [(4001, 60), (4002, 130), (4003, 300), (4004, 700)]:
        extra_u.append(np.full(deg, hub))
        extra_v.append(rng.choice(np.setdiff1d(np.arange(n), [hub]), deg, replace=False))
    eu, ev = synth.graphs._canonical_unique(np.concatenate([eu, *extra_u]), np.concatenate([ev, *extra_v]), n)
    g = synth.csr_from_edges(n, eu, ev, rng.uniform(0.5, 2, size=len(eu)))
    X, Y = rng.random((12, n)), rng.random((12, n))
    want = ocg.ge_d2_cg(g.n, g.rowptr, g.colidx, g.w, X, Y, rtol=1e-13)[0]
    return g, X, Y, want


@pytest.mark.parametrize("row_max_pct", [10, 50, 100, 200, 1000])
@pytest.mark.parametrize("blocks_pct", [10, 100, 400])
def test_every_setting_matches_oracle(nvd, hub_graph, row_max_pct, blocks_pct):
    g, X, Y, want = hub_graph
    G = nvd.Graph.from_csr(g)
    G.set_tuning(mode=nvd.MODE_FP64, row_max_pct=row_max_pct, blocks_pct=blocks_pct)
    for kt in (1, 8, 16):
        for fold in (False, True):
            d2 = nvd.ge_distance(G, on(X), on(Y), rtol=1e-12, kt=kt, fold_direction=fold)
            assert rel(d2.cpu().numpy(), want) < 1e-8, (kt, fold, row_max_pct, blocks_pct)
    d2 = nvd.ge_distance(G, on(X), on(Y), mode=nvd.MODE_FP32, rtol=1e-7, kt=32)
    assert rel(d2.cpu().numpy(), want) < 1e-4
    d2 = nvd.ge_distance(G, on(X), on(Y), mode=nvd.MODE_MIXED, rtol=1e-5, d2_rtol=1e-10, kt=16,
                         fold_direction=True)
    assert rel(d2.cpu().numpy(), want) < 1e-8


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_tune_then_solve(nvd, hub_graph, mode):
    g, X, Y, want = hub_graph
    G = nvd.Graph.from_csr(g)
    r = G.tune(mode=mode, k=12)
    assert r["kt"] in (1, 4, 8, 16, 32) and (mode != 0 or r["kt"] <= 16)
    assert r["row_max_pct"] in (50, 100, 200) and r["blocks_pct"] in (25, 50, 100, 200)
    assert r["persistent"] in (0, 1) and (mode != 2 or r["persistent"] == 0)
    assert r["fold_direction"] in (0, 1)
    assert r["candidates"] >= 5 and r["ms_per_iter"] > 0
    tol = {0: 1e-8, 1: 1e-4, 2: 1e-8}[mode]
    kw = dict(mode=mode, rtol={0: 1e-12, 1: 1e-7, 2: 1e-6}[mode])
    if mode == 2:
        kw["d2_rtol"] = 1e-10
    a = nvd.ge_distance(G, on(X), on(Y), **kw)
    assert rel(a.cpu().numpy(), want) < tol
    # the tuned tile width and launch mode are what an open call uses
    b = nvd.ge_distance(G, on(X), on(Y), kt=r["kt"], persistent=bool(r["persistent"]),
                        fold_direction=bool(r["fold_direction"]), **kw)
    assert torch.equal(a, b)


def test_tune_single_rhs_small_graph(nvd):
    wl = synth.workload_ba_small()
    g = wl.graph
    X, Y = wl.pairs(0, 4)
    want = dense.ge_d2_eig(g.n, g.rowptr, g.colidx, g.w, X, Y)
    G = nvd.Graph.from_csr(g)
    r = G.tune(mode=nvd.MODE_FP64, k=4, single_rhs=True)
    assert r["kt"] == 1
    d2 = nvd.ge_distance(G, on(X), on(Y), rtol=1e-10, single_rhs=True)
    assert rel(d2.cpu().numpy(), want) < 1e-8
