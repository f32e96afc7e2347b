"""Host side of the exact degree-1/2 elimination (nvd_eliminate_host, no GPU work):
the reduced graph must be the Schur complement of the Laplacian onto the kept
nodes (dense check), with every kept node of degree >= 3 or the last node of its
component, and chains must go in a logarithmic number of rounds."""
import ctypes

import numpy as np
import pytest

import synth
from oracle import dense


@pytest.fixture(scope="module")
def lib():
    from paper_2310_11222_gb300 import build
    build.build()
    import paper_2310_11222_gb300 as nvd
    return nvd.load_library()


def eliminate(lib, g):
    n, nnz = g.n, int(g.rowptr[-1])
    rp = np.ascontiguousarray(g.rowptr, np.int64)
    ci = np.ascontiguousarray(g.colidx, np.int32)
    w = np.ascontiguousarray(g.w, np.float64)
    nk, rounds = ctypes.c_int64(0), ctypes.c_int32(0)
    keep = np.zeros(n, np.int32)
    rrp = np.zeros(n + 1, np.int64)
    rci = np.zeros(max(nnz, 1), np.int32)
    rw = np.zeros(max(nnz, 1))
    rc = lib.nvd_eliminate_host(ctypes.c_int64(n), rp.ctypes.data, ci.ctypes.data, w.ctypes.data, ctypes.byref(nk),
                                keep.ctypes.data, rrp.ctypes.data, rci.ctypes.data, rw.ctypes.data,
                                ctypes.byref(rounds))
    assert rc == 0
    K = nk.value
    return keep[:K], rrp[:K + 1], rci[:rrp[K]], rw[:rrp[K]], rounds.value


def schur_check(g, keep, rrp, rci, rw):
    L = dense.laplacian_dense(g.n, g.rowptr, g.colidx, g.w)
    E = np.setdiff1d(np.arange(g.n), keep)
    S = L[np.ix_(keep, keep)]
    if len(E):
        S = S - L[np.ix_(keep, E)] @ np.linalg.solve(L[np.ix_(E, E)], L[np.ix_(E, keep)])
    K = len(keep)
    Lr = np.zeros((K, K))
    for i in range(K):
        for e in range(rrp[i], rrp[i + 1]):
            assert rci[e] != i
            Lr[i, rci[e]] -= rw[e]
            Lr[i, i] += rw[e]
    A = csr_dense(K, rrp, rci, rw)
    assert np.array_equal(A, A.T)          # bitwise: w_ac and w_ca merged in the same order
    assert np.max(np.abs(S - Lr)) <= 1e-12 * max(1.0, np.max(np.abs(L)))
    return Lr


def weighted(g, seed):
    rng = np.random.default_rng(seed)
    return synth.csr_from_edges(g.n, g.eu, g.ev, rng.uniform(0.5, 2.0, g.m))


@pytest.mark.parametrize("model,deg", [("er", 2), ("er", 4), ("ws", 2), ("ws", 4), ("ba", 2), ("ba", 4), ("sbm", 2)])
def test_reduced_graph_is_the_schur_complement(lib, model, deg):
    g = weighted(synth.sweep_graph(model, 300, deg, seed=deg + 7), deg)
    keep, rrp, rci, rw, _ = eliminate(lib, g)
    Lr = schur_check(g, keep, rrp, rci, rw)
    # every kept node has >= 3 neighbours in the reduced graph, or is alone in its component
    comp, _ = dense.components(g.n, g.rowptr, g.colidx)
    deg_red = np.diff(rrp)
    per_comp = np.bincount(comp[keep], minlength=comp.max() + 1)
    assert np.all((deg_red >= 3) | (per_comp[comp[keep]] == 1))
    assert np.all(np.diag(Lr) >= 0)


def test_trees_and_paths_reduce_to_one_node_in_few_rounds(lib):
    rng = np.random.default_rng(3)
    for n in (2, 17, 300, 4096):
        g = synth.csr_from_edges(n, *synth.path_graph(n), rng.uniform(0.5, 2.0, n - 1))
        keep, rrp, _, _, rounds = eliminate(lib, g)
        assert len(keep) == 1 and rrp[-1] == 0
        assert rounds <= 2 * int(np.ceil(np.log2(n))) + 2
    pu, cv = synth.random_tree(500, rng)
    t = synth.csr_from_edges(500, pu, cv, rng.uniform(0.5, 2.0, 499))
    keep, rrp, _, _, _ = eliminate(lib, t)
    assert len(keep) == 1


def test_series_rule_and_untouched_dense_core(lib):
    # a cycle: series reductions leave two nodes joined by two parallel conductances,
    # i.e. one neighbour each, and the last leaf goes too
    n = 9
    w = np.arange(1, n + 1, dtype=float)
    g = synth.csr_from_edges(n, *synth.cycle_graph(n), w)
    keep, rrp, rci, rw, _ = eliminate(lib, g)
    schur_check(g, keep, rrp, rci, rw)
    assert len(keep) == 1
    # a cycle with one chord between opposite nodes keeps the chord's end points:
    # after the series rule they are joined by three parallel paths (one neighbour
    # each), so they go as well
    eu, ev = synth.cycle_graph(8)
    g = synth.csr_from_edges(8, np.append(eu, 0), np.append(ev, 4), np.arange(1, 10, dtype=float))
    keep, rrp, rci, rw, _ = eliminate(lib, g)
    schur_check(g, keep, rrp, rci, rw)
    assert len(keep) == 1
    # K_5 has no node of degree <= 2: nothing is eliminated
    k5 = synth.csr_from_edges(5, *synth.complete_graph(5), np.ones(10))
    keep, rrp, rci, rw, rounds = eliminate(lib, k5)
    assert len(keep) == 5 and rounds == 0
    schur_check(k5, keep, rrp, rci, rw)


def test_disconnected_with_isolated_nodes(lib):
    rng = np.random.default_rng(9)
    parts = [synth.csr_from_edges(30, *synth.path_graph(30), np.ones(29)),
             synth.csr_from_edges(6, *synth.complete_graph(6), rng.uniform(0.5, 2.0, 15)),
             synth.csr_from_edges(12, *synth.star_graph(11), rng.uniform(0.5, 2.0, 11))]
    u, _ = synth.disjoint_union(parts)
    g = synth.csr_from_edges(u.n + 3, u.eu, u.ev, u.ew)
    keep, rrp, rci, rw, _ = eliminate(lib, g)
    schur_check(g, keep, rrp, rci, rw)
    # path -> 1 node, K_6 -> 6, star -> 1, isolated nodes stay
    assert len(keep) == 1 + 6 + 1 + 3


def test_invalid_arguments(lib):
    assert lib.nvd_eliminate_host(ctypes.c_int64(0), None, None, None, None, None, None, None, None, None) == 1


def program(lib, g):
    n = g.n
    rp = np.ascontiguousarray(g.rowptr, np.int64)
    ci = np.ascontiguousarray(g.colidx, np.int32)
    w = np.ascontiguousarray(g.w, np.float64)
    cnt = np.zeros(5, np.int64)
    null = [None] * 14
    assert lib.nvd_eliminate_host_program(ctypes.c_int64(n), rp.ctypes.data, ci.ctypes.data, w.ctypes.data,
                                          cnt.ctypes.data, *null) == 0
    R, K, NR, NK, T = (int(v) for v in cnt)
    a = dict(rec_v=np.zeros(max(R, 1), np.int32), rec_d=np.zeros(max(R, 1)), round_ptr=np.zeros(T + 1, np.int64),
             rin_ptr=np.zeros(R + 1, np.int64), rin_src=np.zeros(max(NR, 1), np.int32), rin_f=np.zeros(max(NR, 1)),
             keep=np.zeros(K, np.int32), kin_ptr=np.zeros(K + 1, np.int64), kin_src=np.zeros(max(NK, 1), np.int32),
             kin_f=np.zeros(max(NK, 1)), rec_t0=np.zeros(max(R, 1), np.int32), rec_t1=np.zeros(max(R, 1), np.int32),
             rec_f0=np.zeros(max(R, 1)), rec_f1=np.zeros(max(R, 1)))
    assert lib.nvd_eliminate_host_program(ctypes.c_int64(n), rp.ctypes.data, ci.ctypes.data, w.ctypes.data,
                                          cnt.ctypes.data, *[a[k].ctypes.data for k in a]) == 0
    return R, K, T, a


def forward(R, K, T, a, b):
    """The device forward pass, round by round, written out."""
    rb = np.zeros(R)
    for t in range(T):
        for r in range(a["round_ptr"][t], a["round_ptr"][t + 1]):
            e0, e1 = a["rin_ptr"][r], a["rin_ptr"][r + 1]
            rb[r] = b[a["rec_v"][r]] + np.dot(a["rin_f"][e0:e1], rb[a["rin_src"][e0:e1]])
    bk = np.array([b[a["keep"][i]] + np.dot(a["kin_f"][a["kin_ptr"][i]:a["kin_ptr"][i + 1]],
                                             rb[a["kin_src"][a["kin_ptr"][i]:a["kin_ptr"][i + 1]]])
                   for i in range(K)])
    return bk, (float(np.sum(rb ** 2 / a["rec_d"][:R])) if R else 0.0), rb


def backward(n, R, K, T, a, rb, zk):
    """The device back-substitution, last round first, written out."""
    z = np.zeros(n)
    z[a["keep"]] = zk
    for t in range(T - 1, -1, -1):
        for r in range(a["round_ptr"][t], a["round_ptr"][t + 1]):
            v = rb[r] / a["rec_d"][r] + a["rec_f0"][r] * z[a["rec_t0"][r]]
            if a["rec_t1"][r] >= 0:
                v += a["rec_f1"][r] * z[a["rec_t1"][r]]
            z[a["rec_v"][r]] = v
    return z


@pytest.mark.parametrize("model,deg", [("er", 2), ("ws", 2), ("ba", 2), ("sbm", 2), ("er", 4)])
def test_program_gives_the_full_graph_d2(lib, model, deg):
    """d^2 of the full graph (dense oracle) = reduced graph's d^2 of the forward-passed
    right-hand side + sum b_r^2 / d_r, for pairs projected per component; and no
    record gathers from a record of its own or a later round (the rounds are the
    parallel steps of the device pass)."""
    g = weighted(synth.sweep_graph(model, 300, deg, seed=deg + 3), deg + 1)
    R, K, T, a = program(lib, g)
    assert R + K == g.n
    rnd = np.zeros(max(R, 1), np.int64)
    for t in range(T):
        rnd[a["round_ptr"][t]:a["round_ptr"][t + 1]] = t
    for r in range(R):
        src = a["rin_src"][a["rin_ptr"][r]:a["rin_ptr"][r + 1]]
        assert np.all(rnd[src] < rnd[r])
    keep, rrp, rci, rw, _ = eliminate(lib, g)
    assert np.array_equal(keep, a["keep"])
    red = synth.csr_from_edges(K, *np.nonzero(np.triu(csr_dense(K, rrp, rci, rw)))[::1],
                               csr_dense(K, rrp, rci, rw)[np.nonzero(np.triu(csr_dense(K, rrp, rci, rw)))]) \
        if rrp[-1] else None
    rng = np.random.default_rng(deg)
    X, Y = rng.random((4, g.n)), rng.random((4, g.n))
    want = dense.ge_d2_eig(g.n, g.rowptr, g.colidx, g.w, X, Y)
    comp, c = dense.components(g.n, g.rowptr, g.colidx)
    zwant = dense.ge_z_dense(g.n, g.rowptr, g.colidx, g.w, X, Y)
    for j in range(4):
        b = dense.project_mean_zero(X[j] - Y[j], comp, c)
        bk, extra, rb = forward(R, K, T, a, b)
        d2_red = 0.0 if red is None else float(dense.ge_d2_eig(K, red.rowptr, red.colidx, red.w,
                                                               bk[None], np.zeros((1, K)))[0])
        assert d2_red + extra == pytest.approx(want[j], rel=1e-10)
        # z: reduced solution on the kept nodes, back-substitution, mean-zero per component
        zk = np.zeros(K) if red is None else dense.ge_z_dense(K, red.rowptr, red.colidx, red.w, bk[None],
                                                              np.zeros((1, K)))[0]
        z = dense.project_mean_zero(backward(g.n, R, K, T, a, rb, zk), comp, c)
        assert np.max(np.abs(z - zwant[j])) <= 1e-9 * np.max(np.abs(zwant[j]))


def csr_dense(K, rrp, rci, rw):
    A = np.zeros((K, K))
    for i in range(K):
        A[i, rci[rrp[i]:rrp[i + 1]]] = rw[rrp[i]:rrp[i + 1]]
    return A


def test_random_small_graphs_property(lib):
    """Hypothesis: random weighted graphs on up to 14 nodes (any density, isolated
    nodes, several components): the reduced graph is the Schur complement and the
    program reproduces the dense d^2."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    @hyp.settings(max_examples=150, deadline=None, derandomize=True)
    @hyp.given(st.integers(2, 14), st.floats(0.05, 0.9), st.integers(0, 2 ** 31 - 1))
    def check(n, p, seed):
        rng = np.random.default_rng(seed)
        eu, ev = synth.random_gnp_small(n, p, rng)
        g = synth.csr_from_edges(n, eu, ev, rng.uniform(0.3, 3.0, len(eu)))
        keep, rrp, rci, rw, _ = eliminate(lib, g)
        schur_check(g, keep, rrp, rci, rw)
        R, K, T, a = program(lib, g)
        comp, c = dense.components(g.n, g.rowptr, g.colidx)
        X, Y = rng.random((1, n)), rng.random((1, n))
        want = dense.ge_d2_eig(g.n, g.rowptr, g.colidx, g.w, X, Y)[0]
        b = dense.project_mean_zero(X[0] - Y[0], comp, c)
        bk, extra, _ = forward(R, K, T, a, b)
        A = csr_dense(K, rrp, rci, rw)
        if rrp[-1]:
            iu = np.nonzero(np.triu(A))
            red = synth.csr_from_edges(K, iu[0], iu[1], A[iu])
            d2r = float(dense.ge_d2_eig(K, red.rowptr, red.colidx, red.w, bk[None], np.zeros((1, K)))[0])
        else:
            d2r = 0.0
        assert d2r + extra == pytest.approx(want, rel=1e-9, abs=1e-12)

    check()
