"""Effective resistance R(u, v) = (e_u - e_v)^T L^+ (e_u - e_v) on node-id pairs,
through the C ABI (nvd_effective_resistance), against closed forms, the dense
oracle and the C CG oracle.

The node-id path builds the indicator right-hand sides inside the delta kernel,
so it must give the GE distance of the indicator vectors (Section 3.1): +inf
across components, 0 on the diagonal.  Tolerances as in test_gpu_parity: FP64
1e-8, MIXED 1e-8, FP32 1e-4 relative.
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
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


@pytest.fixture(scope="module")
def union_case():
    """Weighted random tree (300), unit cycle C_301, unit path P_200, K_50 with weight
    1.7, a star with 40 weighted leaves and 5 isolated nodes, node labels shuffled
    (so the internal component order differs from the user's); 37 pairs with
    closed-form resistances, including u = v and pairs across components."""
    rng = np.random.default_rng(77)
    pu, cv = synth.random_tree(300, rng)
    tw = rng.uniform(0.4, 2.5, size=len(pu))
    sw = rng.uniform(0.5, 3.0, size=40)
    parts = [synth.csr_from_edges(300, pu, cv, tw),
             synth.csr_from_edges(301, *synth.cycle_graph(301), np.ones(301)),
             synth.csr_from_edges(200, *synth.path_graph(200), np.ones(199)),
             synth.csr_from_edges(50, *synth.complete_graph(50), np.full(50 * 49 // 2, 1.7)),
             synth.csr_from_edges(41, *synth.star_graph(40), sw)]
    u0, offs = synth.disjoint_union(parts)
    n = u0.n + 5
    lab = rng.permutation(n)                                    # user label of each union node
    g = synth.csr_from_edges(n, lab[u0.eu], lab[u0.ev], u0.ew)
    T, C, P, K, S, I = offs[0], offs[1], offs[2], offs[3], offs[4], offs[5]

    def tree_r(i, j):                                           # sum of 1/w along the tree path
        par = {int(c): (int(p), w) for p, c, w in zip(pu, cv, tw)}
        anc = {}
        x, acc = i, 0.0
        while True:
            anc[x] = acc
            if x not in par:
                break
            acc += 1.0 / par[x][1]
            x = par[x][0]
        x, acc = j, 0.0
        while x not in anc:
            acc += 1.0 / par[x][1]
            x = par[x][0]
        return acc + anc[x]

    pairs = []
    for i, j in [(0, 299), (17, 250), (123, 5), (42, 43)]:
        pairs.append((T + i, T + j, tree_r(i, j)))
    for h in [1, 2, 50, 150, 151, 300]:
        pairs.append((C, C + h, h * (301 - h) / 301))
    for a, b in [(0, 199), (10, 20), (199, 198)]:
        pairs.append((P + a, P + b, float(abs(a - b))))
    for a, b in [(0, 1), (7, 49), (30, 12)]:
        pairs.append((K + a, K + b, 2.0 / (50 * 1.7)))
    for a, b in [(1, 2), (5, 40), (0, 13)]:
        want = (1 / sw[a - 1] if a else 0.0) + 1 / sw[b - 1]
        pairs.append((S + a, S + b, want))
    for a, b in [(T + 3, T + 3), (C + 7, C + 7), (I, I)]:
        pairs.append((a, b, 0.0))
    for a, b in [(T + 1, C + 1), (P + 4, K + 9), (S, T), (I, I + 1), (I + 2, C), (K + 3, I + 4)]:
        pairs.append((a, b, np.inf))
    while len(pairs) < 37:                                       # more in-component pairs
        a, b = rng.integers(0, 300, 2)
        if a != b:
            pairs.append((T + a, T + b, tree_r(int(a), int(b))))
    U = lab[np.array([p[0] for p in pairs])]
    V = lab[np.array([p[1] for p in pairs])]
    want = np.array([p[2] for p in pairs])
    return g, U, V, want


def check(R, want, tol):
    fin = np.isfinite(want)
    assert np.array_equal(np.isposinf(R), np.isposinf(want))
    assert np.all(R[want == 0.0] == 0.0)
    nz = fin & (want > 0)
    assert rel(R[nz], want[nz]) < tol


def test_union_closed_forms_and_dense_oracle(nvd, union_case):
    g, U, V, want = union_case
    ref = dense.effective_resistance(g.n, g.rowptr, g.colidx, g.w, U, V)
    check(ref, want, 1e-10)                                      # the oracle agrees with the closed forms
    G = nvd.Graph.from_csr(g)
    R, st = nvd.effective_resistance(G, U, V, rtol=1e-11, return_stats=True)
    check(R, want, 1e-8)
    check(R, ref, 1e-8)
    solved = np.isfinite(want) & (want > 0)
    assert all(s["status"] == 0 for s in st)
    assert all((s["iters"] > 0) == bool(f) for s, f in zip(st, solved))


@pytest.mark.parametrize("kt", [1, 4, 8, 16, 32])
@pytest.mark.parametrize("persistent", [False, True])
def test_union_every_tile_width(nvd, union_case, kt, persistent):
    g, U, V, want = union_case
    G = nvd.Graph.from_csr(g)
    R = nvd.effective_resistance(G, U, V, rtol=1e-11, kt=kt, persistent=persistent)
    check(R, want, 1e-8)


def test_union_fp32_and_mixed(nvd, union_case):
    g, U, V, want = union_case
    G = nvd.Graph.from_csr(g)
    check(nvd.effective_resistance(G, U, V, mode=nvd.MODE_FP32, rtol=1e-6), want, 1e-4)
    check(nvd.effective_resistance(G, U, V, mode=nvd.MODE_MIXED, rtol=1e-4, d2_rtol=1e-11), want, 1e-8)


def test_union_d2_stop(nvd, union_case):
    """The d^2 stop on node-id pairs: every resistance within its d2_rtol (1e-6) of the
    closed forms, single right-hand side and tiles of 8."""
    g, U, V, want = union_case
    G = nvd.Graph.from_csr(g)
    for kw in (dict(kt=1), dict(kt=8)):
        R, st = nvd.effective_resistance(G, U, V, rtol=1e-12, d2_stop=True, d2_rtol=1e-6, return_stats=True, **kw)
        check(R, want, 1e-6)
        assert all(s["status"] == 0 for s in st)


def test_equals_ge_distance_of_indicators(nvd):
    """On the BA workload graph: the node-id path and nvd_ge_distance on the dense
    indicator vectors run the same solve."""
    g = synth.workload_ba_small().graph
    rng = np.random.default_rng(3)
    U = rng.integers(0, g.n, 40)
    V = (U + 1 + rng.integers(0, g.n - 1, 40)) % g.n
    X = np.zeros((40, g.n)); Y = np.zeros((40, g.n))
    X[np.arange(40), U] = 1.0
    Y[np.arange(40), V] = 1.0
    G = nvd.Graph.from_csr(g)
    R = nvd.effective_resistance(G, U, V, rtol=1e-11, kt=16)
    d2 = nvd.ge_distance(G, torch.as_tensor(X, device=DEV), torch.as_tensor(Y, device=DEV), rtol=1e-11,
                         kt=16).cpu().numpy()
    assert rel(R, d2) < 1e-13
    assert rel(R, dense.effective_resistance(g.n, g.rowptr, g.colidx, g.w, U, V)) < 1e-8


def test_foster_on_er_with_components(nvd):
    """ER G(n = 3000, m = 4500) keeps several components and isolated nodes; with
    lognormal weights, sum over edges of w_e R_e = n - c (Foster's theorem)."""
    rng = np.random.default_rng(11)
    eu, ev = synth.erdos_renyi_gnm(3000, 4500, rng)
    w = rng.lognormal(0.0, 0.5, size=len(eu))
    g = synth.csr_from_edges(3000, eu, ev, w)
    _, c = ocg.components(g.n, g.rowptr, g.colidx)
    assert c > 10
    G = nvd.Graph.from_csr(g)
    R = nvd.effective_resistance(G, g.eu, g.ev, rtol=1e-12)
    assert np.all(np.isfinite(R)) and np.all(R > 0)
    assert abs(float(np.sum(g.ew * R)) - (g.n - c)) <= 1e-8 * (g.n - c)


def test_empty_and_invalid_ids(nvd, union_case):
    g, U, V, _ = union_case
    G = nvd.Graph.from_csr(g)
    assert nvd.effective_resistance(G, [], []).shape == (0,)
    for bad in ([-1], [g.n]):
        with pytest.raises(nvd.NvdError) as e:
            nvd.effective_resistance(G, bad, [0])
        assert e.value.status == 1
    with pytest.raises(ValueError):
        nvd.effective_resistance(G, [0, 1], [2])


@pytest.mark.slow
def test_er_large_full_size_sampled(nvd):
    """ER n = 1e6 (largest component), the graph the bench times: 12 seeded node pairs
    in FP64 against the C FP64 CG oracle on the indicator vectors."""
    g = synth.workload_er_large().graph
    rng = np.random.default_rng(19)
    U = rng.integers(0, g.n, 12)
    V = (U + 1 + rng.integers(0, g.n - 1, 12)) % g.n
    X = np.zeros((12, g.n)); Y = np.zeros((12, g.n))
    X[np.arange(12), U] = 1.0
    Y[np.arange(12), V] = 1.0
    want, it, _ = ocg.ge_d2_cg(g.n, g.rowptr, g.colidx, g.w, X, Y, rtol=1e-12)
    assert np.all(it > 0)
    G = nvd.Graph.from_csr(g)
    R, st = nvd.effective_resistance(G, U, V, rtol=1e-10, return_stats=True)
    assert rel(R, want) < 1e-8
    assert all(s["status"] == 0 for s in st)


# ------------------------------------------------- effective-resistance matrix

def oracle_matrix(g, nodes):
    a, b = np.meshgrid(nodes, nodes, indexing="ij")
    return dense.effective_resistance(g.n, g.rowptr, g.colidx, g.w, a.ravel(), b.ravel()).reshape(len(nodes), -1)


def check_matrix(R, want, tol):
    assert R.shape == want.shape
    assert np.array_equal(np.isposinf(R), np.isposinf(want))
    assert np.all(R[want == 0.0] == 0.0)
    nz = np.isfinite(want) & (want > 0)
    assert rel(R[nz], want[nz]) < tol


@pytest.mark.parametrize("kt", [1, 16])
def test_matrix_on_union_subset(nvd, union_case, kt):
    """30 subset nodes drawn from every component of the shuffled union, with
    repeats and isolated nodes, against the dense oracle entry by entry."""
    g = union_case[0]
    rng = np.random.default_rng(5)
    nodes = rng.choice(g.n, 26, replace=False)
    nodes = np.concatenate([nodes, nodes[[0, 3]], nodes[[7, 7]]])
    rng.shuffle(nodes)
    want = oracle_matrix(g, nodes)
    assert np.isinf(want).any() and np.isfinite(want[want > 0]).any()
    G = nvd.Graph.from_csr(g)
    R, st = nvd.resistance_matrix(G, nodes, rtol=1e-12, kt=kt, return_stats=True)
    check_matrix(R, want, 1e-8)
    assert all(s["status"] == 0 for s in st)
    Rp = nvd.resistance_matrix(G, nodes, rtol=1e-12, kt=kt, persistent=True)
    check_matrix(Rp, want, 1e-8)


def test_matrix_edge_cases(nvd, union_case):
    g = union_case[0]
    G = nvd.Graph.from_csr(g)
    assert nvd.resistance_matrix(G, []).shape == (0, 0)
    assert np.array_equal(nvd.resistance_matrix(G, [4]), np.zeros((1, 1)))
    assert np.array_equal(nvd.resistance_matrix(G, [4, 4]), np.zeros((2, 2)))
    for bad in ([-1, 0], [0, g.n]):
        with pytest.raises(nvd.NvdError) as e:
            nvd.resistance_matrix(G, bad)
        assert e.value.status == 1


@pytest.mark.slow
def test_matrix_er_large_full_size(nvd):
    """300 seeded nodes of the n = 1e6 ER graph: 299 solves, run in two batches of
    z (268 + 31 columns at 2^28 doubles per batch).  Zero diagonal, symmetry, the
    triangle inequality on sampled triples, 40 sampled entries against the direct
    per-pair path and 3 against the C FP64 CG oracle."""
    g = synth.workload_er_large().graph
    rng = np.random.default_rng(29)
    nodes = rng.choice(g.n, 300, replace=False)
    G = nvd.Graph.from_csr(g)
    R = nvd.resistance_matrix(G, nodes, rtol=1e-11)
    assert np.all(np.diag(R) == 0.0) and np.all(np.isfinite(R))
    off = ~np.eye(300, dtype=bool)
    assert np.all(R[off] > 0)
    assert np.max(np.abs(R - R.T)[off] / R[off]) < 1e-8
    i, j, k = rng.integers(0, 300, (3, 2000))
    assert np.all(R[i, k] <= R[i, j] + R[j, k] + 1e-9)
    a, b = rng.integers(0, 300, (2, 40))
    a, b = a[a != b], b[a != b]
    direct = nvd.effective_resistance(G, nodes[a], nodes[b], rtol=1e-11)
    assert rel(R[a, b], direct) < 1e-8
    X = np.zeros((3, g.n)); Y = np.zeros((3, g.n))
    X[np.arange(3), nodes[a[:3]]] = 1.0
    Y[np.arange(3), nodes[b[:3]]] = 1.0
    want, it, _ = ocg.ge_d2_cg(g.n, g.rowptr, g.colidx, g.w, X, Y, rtol=1e-12)
    assert np.all(it > 0)
    assert rel(R[a[:3], b[:3]], want) < 1e-8


# ------------------------------------------------------------ network variance

def test_network_variance(nvd):
    """Uniform distributions on a unit cycle C_301 and on K_50 (weight 1.7) inside
    one graph with labels shuffled: tr(L^+)/n = (n^2 - 1)/(12 n) and (n - 1)/(n^2 w);
    random distributions on a weighted BA graph against the dense oracle; a point
    mass gives 0 and mass on two components gives inf."""
    cyc = synth.csr_from_edges(301, *synth.cycle_graph(301), np.ones(301))
    kn = synth.csr_from_edges(50, *synth.complete_graph(50), np.full(50 * 49 // 2, 1.7))
    u0, offs = synth.disjoint_union([cyc, kn])
    rng = np.random.default_rng(8)
    lab = rng.permutation(u0.n)
    g = synth.csr_from_edges(u0.n, lab[u0.eu], lab[u0.ev], u0.ew)
    G = nvd.Graph.from_csr(g)
    v = nvd.network_variance(G, lab[np.arange(301)], np.full(301, 1 / 301), rtol=1e-12)
    assert v == pytest.approx((301 ** 2 - 1) / (12 * 301), rel=1e-8)
    v = nvd.network_variance(G, lab[301 + np.arange(50)], np.full(50, 1 / 50), rtol=1e-12)
    assert v == pytest.approx(49 / (2500 * 1.7), rel=1e-8)
    assert nvd.network_variance(G, [lab[5]], [1.0]) == 0.0
    assert nvd.network_variance(G, [lab[5], lab[310]], [0.5, 0.5]) == np.inf
    assert nvd.network_variance(G, [lab[5], lab[310]], [1.0, 0.0]) == 0.0
    for bad_nodes, bad_p in (([0, 1], [0.5, -0.5]), ([0, g.n], [1.0, 0.0])):
        with pytest.raises(nvd.NvdError) as e:
            nvd.network_variance(G, bad_nodes, bad_p)
        assert e.value.status == 1
    b = synth.workload_ba_small().graph
    bw = synth.csr_from_edges(b.n, b.eu, b.ev, rng.uniform(0.5, 2.0, b.m))
    B = nvd.Graph.from_csr(bw)
    for t in range(3):
        nodes = rng.choice(bw.n, 40, replace=False)
        p = rng.dirichlet(np.ones(40))
        want = dense.network_variance(bw.n, bw.rowptr, bw.colidx, bw.w, nodes, p)
        assert nvd.network_variance(B, nodes, p, rtol=1e-12) == pytest.approx(want, rel=1e-8)
