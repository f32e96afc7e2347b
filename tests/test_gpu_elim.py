"""Solves on the reduced graph after exact degree-1/2 elimination
(nvd_graph_eliminate + NVD_SOLVE_ELIMINATE): d^2 must match the oracle on the full
graph (FP64 1e-8, FP32 1e-4, MIXED 1e-8) and z_out (back-substitution) the dense
oracle's z, including disconnected graphs with isolated nodes in a shuffled node
order, with fewer PCG iterations on the sparse families where Jacobi PCG is slow
(none at all once a graph reduces to one node per component)."""
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


def on(a):
    return torch.as_tensor(a, dtype=torch.float64, device=DEV)


def weighted(g, seed):
    rng = np.random.default_rng(seed)
    return synth.csr_from_edges(g.n, g.eu, g.ev, rng.uniform(0.5, 2.0, g.m))


@pytest.fixture(scope="module")
def families():
    out = []
    for model, deg in [("ws", 2), ("ba", 2), ("er", 2), ("er", 4), ("sbm", 2)]:
        g = weighted(synth.sweep_graph(model, 10000, deg, seed=deg + 11), deg)
        X, Y = synth.sparse_uniform_pairs(g.n, 8, 0.10, 31)
        # the WS ring of degree 2 has an FP64 residual floor near 2e-11
        want, it, _ = ocg.ge_d2_cg(g.n, g.rowptr, g.colidx, g.w, X, Y, rtol=1e-11 if model == "ws" else 1e-13)
        assert np.all(it > 0)
        out.append((f"{model}{deg}", g, X, Y, want))
    return out


@pytest.mark.parametrize("kw", [dict(single_rhs=True), dict(kt=8)])
def test_sparse_families_match_the_oracle_with_fewer_iterations(nvd, families, kw):
    for name, g, X, Y, want in families:
        G = nvd.Graph.from_csr(g)
        info = G.eliminate()
        assert info["n_kept"] + info["n_eliminated"] == g.n
        d2, st = nvd.ge_distance(G, on(X), on(Y), rtol=1e-11, eliminate=True, return_stats=True, **kw)
        assert rel(d2.cpu().numpy(), want) < 1e-8, name
        assert all(s["status"] == 0 for s in st)
        if name in ("ws2", "ba2"):
            # every component reduces to one node: no PCG at all (Jacobi PCG on the
            # full graph needs ~1,000 (BA) and ~5,000 (WS) iterations per pair)
            assert info["nnz_kept"] == 0 and all(s["iters"] == 0 for s in st)
        else:
            _, st_full = nvd.ge_distance(G, on(X), on(Y), rtol=1e-11, return_stats=True, **kw)
            assert sum(s["iters"] for s in st) < sum(s["iters"] for s in st_full), name


def test_modes_on_the_reduced_graph(nvd, families):
    name, g, X, Y, want = families[2]                      # ER mean degree 2
    G = nvd.Graph.from_csr(g)
    G.eliminate()
    d32 = nvd.ge_distance(G, on(X), on(Y), mode=nvd.MODE_FP32, rtol=1e-6, eliminate=True)
    assert rel(d32.cpu().numpy(), want) < 1e-4
    dmx = nvd.ge_distance(G, on(X), on(Y), mode=nvd.MODE_MIXED, rtol=1e-4, d2_rtol=1e-11, eliminate=True)
    assert rel(dmx.cpu().numpy(), want) < 1e-8
    dds = nvd.ge_distance(G, on(X), on(Y), rtol=1e-13, d2_stop=True, d2_rtol=1e-8, eliminate=True)
    assert rel(dds.cpu().numpy(), want) < 1e-8


@pytest.mark.parametrize("xdtype", [torch.float64, torch.float32])
def test_shuffled_disconnected_graph_with_isolated_nodes(nvd, xdtype):
    """Trees, a cycle with pendant paths, a dense K_12 core with whiskers and isolated
    nodes, labels shuffled; 13 dense random pairs (ragged tiles) against the dense
    oracle."""
    rng = np.random.default_rng(17)
    pu, cv = synth.random_tree(60, rng)
    parts = [synth.csr_from_edges(60, pu, cv, rng.uniform(0.5, 2.0, 59))]
    eu, ev = synth.cycle_graph(40)
    eu = np.concatenate([eu, [0, 50, 51, 10, 53]])
    ev = np.concatenate([ev, [50, 51, 52, 53, 54]])
    parts.append(synth.csr_from_edges(55, eu, ev, rng.uniform(0.5, 2.0, len(eu))))
    ku, kv = synth.complete_graph(12)
    ku = np.concatenate([ku, [0, 12, 3, 14, 15]])
    kv = np.concatenate([kv, [12, 13, 14, 15, 16]])
    parts.append(synth.csr_from_edges(17, ku, kv, rng.uniform(0.5, 2.0, len(ku))))
    u0, _ = synth.disjoint_union(parts)
    n = u0.n + 5
    lab = rng.permutation(n)
    g = synth.csr_from_edges(n, lab[u0.eu], lab[u0.ev], u0.ew)
    X, Y = rng.random((13, n)), rng.random((13, n))
    G = nvd.Graph.from_csr(g)
    info = G.eliminate()
    assert info["n_kept"] < n
    npdt = np.float32 if xdtype == torch.float32 else np.float64       # the inputs as the GPU sees them
    X64, Y64 = X.astype(npdt).astype(np.float64), Y.astype(npdt).astype(np.float64)
    want = dense.ge_d2_eig(g.n, g.rowptr, g.colidx, g.w, X64, Y64)
    zwant = dense.ge_z_dense(g.n, g.rowptr, g.colidx, g.w, X64, Y64)
    for kw in (dict(single_rhs=True), dict(kt=4)):
        d2, z = nvd.ge_distance(G, torch.as_tensor(X, dtype=xdtype, device=DEV),
                                torch.as_tensor(Y, dtype=xdtype, device=DEV), rtol=1e-12, eliminate=True,
                                return_z=True, **kw)
        assert rel(d2.cpu().numpy(), want) < 1e-8
        # z by back-substitution, mean-zero per component, in the user's node order
        ztol = 1e-6 if xdtype == torch.float32 else 1e-8      # z_out is stored in the dtype of x
        assert np.max(np.abs(z.cpu().numpy().astype(np.float64) - zwant)) <= ztol * np.max(np.abs(zwant))


def test_nothing_to_eliminate_and_invalid_uses(nvd):
    rng = np.random.default_rng(2)
    g = synth.csr_from_edges(30, *synth.complete_graph(30), rng.uniform(0.5, 2.0, 435))
    X, Y = rng.random((4, 30)), rng.random((4, 30))
    G = nvd.Graph.from_csr(g)
    with pytest.raises(nvd.NvdError) as e:                      # no nvd_graph_eliminate yet
        nvd.ge_distance(G, on(X), on(Y), eliminate=True)
    assert e.value.status == 1
    info = G.eliminate()
    assert info["n_eliminated"] == 0 and info["rounds"] == 0
    d2 = nvd.ge_distance(G, on(X), on(Y), rtol=1e-12, eliminate=True).cpu().numpy()
    assert rel(d2, nvd.ge_distance(G, on(X), on(Y), rtol=1e-12).cpu().numpy()) < 1e-10
    with pytest.raises(nvd.NvdError) as e:                      # host inputs
        nvd.ge_distance(G, X, Y, eliminate=True)
    assert e.value.status == 1


def test_effective_resistance_on_the_reduced_graph(nvd):
    """Node-id pairs through the eliminated graph: a weighted tree, a cycle with
    pendant paths and an ER graph of mean degree 3 with isolated nodes, against
    the dense oracle (0 on the diagonal, inf across components)."""
    rng = np.random.default_rng(23)
    pu, cv = synth.random_tree(80, rng)
    eu, ev = synth.cycle_graph(50)
    er_u, er_v = synth.erdos_renyi_gnm(150, 225, rng)
    parts = [synth.csr_from_edges(80, pu, cv, rng.uniform(0.5, 2.0, 79)),
             synth.csr_from_edges(53, np.concatenate([eu, [0, 50, 51]]), np.concatenate([ev, [50, 51, 52]]),
                                  rng.uniform(0.5, 2.0, 53)),
             synth.csr_from_edges(150, er_u, er_v, rng.uniform(0.5, 2.0, len(er_u)))]
    u0, _ = synth.disjoint_union(parts)
    lab = rng.permutation(u0.n)
    g = synth.csr_from_edges(u0.n, lab[u0.eu], lab[u0.ev], u0.ew)
    U = rng.integers(0, g.n, 60)
    V = rng.integers(0, g.n, 60)
    V[:3] = U[:3]
    want = dense.effective_resistance(g.n, g.rowptr, g.colidx, g.w, U, V)
    G = nvd.Graph.from_csr(g)
    G.eliminate()
    R = nvd.effective_resistance(G, U, V, rtol=1e-12, eliminate=True)
    fin = np.isfinite(want)
    assert np.array_equal(np.isinf(R), ~fin)
    assert np.all(R[want == 0] == 0)
    nz = fin & (want > 0)
    assert rel(R[nz], want[nz]) < 1e-8
