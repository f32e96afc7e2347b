"""The multi-column SpMM's four gather engines -- register loads per slice
(GATHER_SLICES), register loads over each warp's step stream (GATHER_STREAM), TMA
tile::gather4 over the stream (GATHER_TMA) and per-lane asynchronous copies over the
stream (GATHER_ACOPY; the last two for tiles whose rows are 64 or 128 bytes) --
against each other and against the oracle: a graph with split heavy rows (degrees up
to 3000), rows on both sides of the light-row limits, several components in a
shuffled node order and isolated nodes, with a ragged last tile.  The three stream
engines run the same plan in the same order (bitwise equal results); every engine
gives each warp a fixed run of work, so its results are bitwise repeatable."""
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


def on(x):
    return torch.as_tensor(x, dtype=torch.float64, device=DEV)


@pytest.fixture(scope="module")
def case():
    rng = np.random.default_rng(21)
    n1 = 6000
    eu, ev = synth.barabasi_albert(n1, 3, rng)
    extra_u = [np.zeros(3000, np.int64)]
    extra_v = [np.arange(1, 3001)]
    for hub, deg in [(4001, 30), (4002, 70), (4003, 129), (4004, 260), (4005, 520), (4006, 1100)]:
        extra_u.append(np.full(deg, hub))
        extra_v.append(rng.choice(np.setdiff1d(np.arange(n1), [hub]), deg, replace=False))
    eu, ev = synth.graphs._canonical_unique(np.concatenate([eu, *extra_u]), np.concatenate([ev, *extra_v]), n1)
    er_u, er_v = synth.erdos_renyi_gnm(1500, 6000, rng)
    er_n, er_u, er_v, _ = synth.largest_component(1500, er_u, er_v)
    n = n1 + er_n + 7                                         # 7 isolated nodes
    lab = rng.permutation(n)
    u = lab[np.concatenate([eu, er_u + n1])]
    v = lab[np.concatenate([ev, er_v + n1])]
    g = synth.csr_from_edges(n, u, v, rng.uniform(0.5, 2.0, len(u)))
    X, Y = rng.random((37, n)), rng.random((37, n))          # 37 pairs: ragged last tile
    want = ocg.ge_d2_cg(g.n, g.rowptr, g.colidx, g.w, X, Y, rtol=1e-13)[0]
    return g, X, Y, want


@pytest.mark.parametrize("mode,kt", [(0, 4), (0, 8), (0, 16), (1, 4), (1, 8), (1, 16), (1, 32), (2, 16),
                                     (2, 32)])
def test_gather_engines_match_each_other_and_the_oracle(nvd, case, mode, kt):
    g, X, Y, want = case
    kw = {0: dict(rtol=1e-12), 1: dict(rtol=1e-7), 2: dict(rtol=1e-5, d2_rtol=1e-11)}[mode]
    tol = {0: 1e-9, 1: 1e-4, 2: 1e-9}[mode]
    tma_ok = kt * (8 if mode == 0 else 4) in (64, 128)
    out = {}
    for gather in (nvd.GATHER_SLICES, nvd.GATHER_STREAM, nvd.GATHER_TMA, nvd.GATHER_ACOPY):
        G = nvd.Graph.from_csr(g)
        G.set_tuning(mode=mode, gather=gather)
        a = nvd.ge_distance(G, on(X), on(Y), mode=mode, kt=kt, **kw)
        assert rel(a.cpu().numpy(), want) < tol, (mode, kt, gather)
        b = nvd.ge_distance(G, on(X), on(Y), mode=mode, kt=kt, **kw)
        assert torch.equal(a, b), (mode, kt, gather)        # fixed work per warp: bitwise repeatable
        out[gather] = a
    # TMA (where the tile allows it, else the register stream again): the same plan,
    # the same sums in the same order
    assert torch.equal(out[nvd.GATHER_STREAM], out[nvd.GATHER_TMA]), tma_ok
    assert torch.equal(out[nvd.GATHER_STREAM], out[nvd.GATHER_ACOPY]), tma_ok
    # per-slice plan: the same CG, rows added in another grouping of the inner products
    assert rel(out[nvd.GATHER_SLICES].cpu().numpy(), out[nvd.GATHER_STREAM].cpu().numpy()) < \
        {0: 1e-10, 1: 1e-5, 2: 1e-10}[mode]


@pytest.mark.parametrize("gather", [1, 2, 3])
@pytest.mark.parametrize("row_max_pct,blocks_pct", [(10, 100), (100, 10), (100, 400), (1000, 100)])
def test_stream_under_other_work_decompositions(nvd, case, gather, row_max_pct, blocks_pct):
    """Few rows per block, very many blocks, and the light-row limit moved so that the
    hub rows land in the sliced layout (long slices) or most rows are chunked."""
    g, X, Y, want = case
    G = nvd.Graph.from_csr(g)
    G.set_tuning(mode=0, row_max_pct=row_max_pct, blocks_pct=blocks_pct, gather=gather)
    d2 = nvd.ge_distance(G, on(X), on(Y), kt=16, rtol=1e-12, fold_direction=True)
    assert rel(d2.cpu().numpy(), want) < 1e-9
    G.set_tuning(mode=1, row_max_pct=row_max_pct, blocks_pct=blocks_pct, gather=gather)
    d2 = nvd.ge_distance(G, on(X), on(Y), mode=1, kt=32, rtol=1e-7)
    assert rel(d2.cpu().numpy(), want) < 1e-4


def test_degree_order_and_l2_window(nvd, case):
    """NVD_GRAPH_REORDER_DEGREE stores each component's nodes by degree (the hub rows
    first): d^2, z in the caller's node order and the weight gradient on the caller's
    entries match the graph in its own order; keeping the hot rows persisting in L2
    changes no result bit."""
    g, X, Y, want = case
    G = nvd.Graph.from_csr(g)
    R = nvd.Graph.from_csr(g, reorder=True)
    for mode, kt, kw, tol in ((0, 16, dict(rtol=1e-12), 1e-9), (1, 32, dict(rtol=1e-7), 1e-4),
                              (2, 32, dict(rtol=1e-5, d2_rtol=1e-11), 1e-9)):
        a, za = nvd.ge_distance(G, on(X), on(Y), mode=mode, kt=kt, return_z=True, **kw)
        outs = []
        for hot in (False, True):
            R.set_tuning(mode=mode, l2_hot=hot)
            b, zb = nvd.ge_distance(R, on(X), on(Y), mode=mode, kt=kt, return_z=True, **kw)
            assert rel(b.cpu().numpy(), want) < tol, (mode, hot)
            assert rel(b.cpu().numpy(), a.cpu().numpy()) < tol
            zs = float(za.abs().max())
            assert float((zb - za).abs().max()) <= (1e-8 if mode != 1 else 1e-3) * zs
            outs.append((b, zb))
        assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    z = nvd.ge_distance(G, on(X), on(Y), rtol=1e-12, return_z=True)[1]
    gw, _, _ = nvd.ge_grad(G, z, on(np.ones(X.shape[0])))
    gr, _, _ = nvd.ge_grad(R, z, on(np.ones(X.shape[0])))
    assert torch.equal(gw, gr)                       # the same sums per caller entry, mapped back
