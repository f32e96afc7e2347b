"""Pins for the oracle: it is checked against facts that do not come from itself.

The GE distance with delta = e_i - e_j is the effective resistance R_ij between
i and j (Section 3.1, GE equation with the Laplacian pseudoinverse), so textbook
closed forms fix it: a path of unit edges has R = n - 1 end to end, the complete
graph has R = 2/n, a tree path has R = sum of 1/w, a cycle has R = h(n-h)/n,
series/parallel rules hold, and Foster's theorem gives sum_e w_e R_e = n - c.
Invariants (metric axioms, shift invariance per component, weight scaling,
permutation invariance) and the agreement of three independent routes (dense
eigendecomposition, grounded Cholesky, C conjugate gradient) complete the pins.
The last tests plant plausible mistakes in copies of the oracle and check that
the pins catch them.
"""
import itertools

import numpy as np
import pytest

import synth
from oracle import dense, cg

ROUTES = ("eig", "grounded", "cg")


def graph(n, eu, ev, ew=None):
    ew = np.ones(len(eu)) if ew is None else np.asarray(ew, dtype=np.float64)
    return synth.csr_from_edges(n, np.asarray(eu), np.asarray(ev), ew)


def d2(g, X, Y, route, rtol=1e-13):
    X = np.atleast_2d(X)
    Y = np.atleast_2d(Y)
    if route == "eig":
        return dense.ge_d2_eig(g.n, g.rowptr, g.colidx, g.w, X, Y)
    if route == "grounded":
        return dense.ge_d2_grounded(g.n, g.rowptr, g.colidx, g.w, X, Y)
    out, it, _ = cg.ge_d2_cg(g.n, g.rowptr, g.colidx, g.w, X, Y, rtol=rtol, threads=2)
    assert np.all(it >= 0)
    return out


def resistance(g, i, j, route, rtol=1e-13):
    x = np.zeros(g.n)
    y = np.zeros(g.n)
    x[i] = 1.0
    y[j] = 1.0
    return float(d2(g, x, y, route, rtol)[0])


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("route", ROUTES)
@pytest.mark.parametrize("n", [2, 5, 31])
def test_unit_path_end_to_end(route, n):
    g = graph(n, *synth.path_graph(n))
    assert resistance(g, 0, n - 1, route) == pytest.approx(n - 1, rel=1e-11)


def test_long_path_cg_only():
    n = 3000
    g = graph(n, *synth.path_graph(n))
    # condition number ~ n^2: a 1e-10 residual target is what FP64 CG reaches here
    assert resistance(g, 0, n - 1, "cg", 1e-10) == pytest.approx(n - 1, rel=1e-9)
    assert resistance(g, 10, 2010, "cg", 1e-10) == pytest.approx(2000, rel=1e-9)


@pytest.mark.parametrize("route", ROUTES)
def test_complete_graph(route):
    n = 9
    wgt = 2.5
    eu, ev = synth.complete_graph(n)
    g = graph(n, eu, ev, np.full(len(eu), wgt))
    # K_n with weight w: L = w (n I - J), so L^+ = P / (n w) and d^2 = |P delta|^2 / (n w)
    assert resistance(g, 2, 7, route) == pytest.approx(2.0 / (n * wgt), rel=1e-11)
    rng = np.random.default_rng(5)
    x, y = rng.random(n), rng.random(n)
    delta = x - y
    pd = delta - delta.mean()
    assert d2(g, x, y, route)[0] == pytest.approx(pd @ pd / (n * wgt), rel=1e-11)


def _tree_path_resistance(parents_u, children_v, weights, i, j):
    """Sum of 1/w along the unique tree path, by walking up parent pointers."""
    parent = {int(c): (int(p), float(wt)) for p, c, wt in zip(parents_u, children_v, weights)}

    def up(a):
        chain = [(a, 0.0)]
        acc = 0.0
        while a in parent:
            p, wt = parent[a]
            acc += 1.0 / wt
            a = p
            chain.append((a, acc))
        return chain

    ci = dict((node, acc) for node, acc in up(i))
    for node, acc in up(j):
        if node in ci:
            return ci[node] + acc
    raise AssertionError("not a tree")


@pytest.mark.parametrize("route", ROUTES)
def test_weighted_tree(route):
    rng = np.random.default_rng(11)
    n = 40
    pu, cv = synth.random_tree(n, rng)
    wts = rng.uniform(0.2, 3.0, size=n - 1)
    g = graph(n, pu, cv, wts)
    for i, j in [(0, 39), (5, 17), (38, 1), (12, 13)]:
        want = _tree_path_resistance(pu, cv, wts, i, j)
        assert resistance(g, i, j, route) == pytest.approx(want, rel=1e-10)


@pytest.mark.parametrize("route", ROUTES)
def test_unit_cycle(route):
    n = 24
    g = graph(n, *synth.cycle_graph(n))
    for h in (1, 5, 12):
        assert resistance(g, 0, h, route) == pytest.approx(h * (n - h) / n, rel=1e-11)


@pytest.mark.parametrize("route", ROUTES)
def test_weighted_cycle_parallel_rule(route):
    rng = np.random.default_rng(3)
    n = 15
    u = np.arange(n)
    v = (u + 1) % n
    wts = rng.uniform(0.5, 2.0, size=n)
    g = graph(n, u, v, wts)
    i, j = 2, 9
    r1 = np.sum(1.0 / wts[i:j])                       # arc i -> j
    r2 = np.sum(1.0 / wts[j:]) + np.sum(1.0 / wts[:i])  # the other arc
    assert resistance(g, i, j, route) == pytest.approx(r1 * r2 / (r1 + r2), rel=1e-11)


@pytest.mark.parametrize("route", ROUTES)
def test_star(route):
    wts = np.array([0.5, 2.0, 4.0, 1.0])
    g = graph(5, *synth.star_graph(4), wts)
    assert resistance(g, 1, 2, route) == pytest.approx(1 / 0.5 + 1 / 2.0, rel=1e-12)
    assert resistance(g, 0, 3, route) == pytest.approx(1 / 4.0, rel=1e-12)
    gu = graph(7, *synth.star_graph(6))
    assert resistance(gu, 3, 6, route) == pytest.approx(2.0, rel=1e-12)


@pytest.mark.parametrize("route", ["eig", "cg"])
def test_foster_theorem(route):
    """sum over edges of w_e R_e = n - c (Foster 1949), also for disconnected graphs."""
    rng = np.random.default_rng(7)
    for n, p in [(12, 0.35), (20, 0.12), (16, 0.5)]:
        eu, ev = synth.random_gnp_small(n, p, rng)
        wts = rng.uniform(0.3, 3.0, size=len(eu))
        g = graph(n, eu, ev, wts)
        _, c = dense.components(g.n, g.rowptr, g.colidx)
        X = np.zeros((len(eu), n))
        Y = np.zeros((len(eu), n))
        X[np.arange(len(eu)), eu] = 1.0
        Y[np.arange(len(eu)), ev] = 1.0
        R = d2(g, X, Y, route)
        assert float(np.sum(wts * R)) == pytest.approx(n - c, rel=1e-10)


def _mixed_union():
    """Weighted tree (12 nodes) + unit cycle C_9 + unit path P_6 + two isolated nodes."""
    rng = np.random.default_rng(41)
    pu, cv = synth.random_tree(12, rng)
    wts = rng.uniform(0.4, 2.5, size=len(pu))
    parts = [graph(12, pu, cv, wts), graph(9, *synth.cycle_graph(9)), graph(6, *synth.path_graph(6))]
    g, offs = synth.disjoint_union(parts)
    g = graph(g.n + 2, g.eu, g.ev, g.ew)                   # nodes g.n, g.n+1 stay isolated
    return g, offs, (pu, cv, wts)


def test_effective_resistance_on_node_pairs():
    """The node-id form: tree path sums, cycle h(n-h)/n and path hop counts inside
    each component, 0 on the diagonal, +inf across components and to isolated nodes."""
    g, offs, (pu, cv, wts) = _mixed_union()
    t0, c0, p0, iso = offs[0], offs[1], offs[2], offs[3]
    U, V, want = [], [], []
    for i, j in [(0, 11), (3, 7), (5, 10)]:
        U.append(t0 + i); V.append(t0 + j); want.append(_tree_path_resistance(pu, cv, wts, i, j))
    for h in range(1, 9):
        U.append(c0); V.append(c0 + h); want.append(h * (9 - h) / 9)
    U.append(p0 + 5); V.append(p0); want.append(5.0)
    U += [c0 + 4, t0 + 2, iso, iso]; V += [c0 + 4, c0 + 1, p0 + 3, iso + 1]; want += [0.0, np.inf, np.inf, np.inf]
    R = dense.effective_resistance(g.n, g.rowptr, g.colidx, g.w, U, V)
    fin = np.isfinite(want)
    assert np.array_equal(np.isinf(R), ~fin)
    assert np.allclose(R[fin], np.asarray(want)[fin], rtol=1e-11, atol=1e-13)
    # the same numbers from the indicator-vector route where the pair is connected
    X = np.zeros((int(fin.sum()), g.n)); Y = np.zeros_like(X)
    X[np.arange(len(X)), np.asarray(U)[fin]] = 1.0
    Y[np.arange(len(Y)), np.asarray(V)[fin]] = 1.0
    assert np.allclose(dense.ge_d2_grounded(g.n, g.rowptr, g.colidx, g.w, X, Y), R[fin], rtol=1e-11, atol=1e-13)


def test_effective_resistance_foster_disconnected():
    """Foster: sum over edges of w_e R(u_e, v_e) = n - c with isolated nodes counted as components."""
    g, _, _ = _mixed_union()
    _, c = dense.components(g.n, g.rowptr, g.colidx)
    R = dense.effective_resistance(g.n, g.rowptr, g.colidx, g.w, g.eu, g.ev)
    assert float(np.sum(g.ew * R)) == pytest.approx(g.n - c, rel=1e-11)


def test_network_variance_pin_catches_dropped_half(monkeypatch):
    """A copy without the factor 1/2 (or with R replaced by R^2) fails the K_n pin."""
    n, wgt = 9, 1.7
    kn = graph(n, *synth.complete_graph(n), np.full(n * (n - 1) // 2, wgt))
    want = (n - 1) / (n * n * wgt)
    orig = dense.effective_resistance
    monkeypatch.setattr(dense, "effective_resistance", lambda *a: 2.0 * orig(*a))
    assert dense.network_variance(kn.n, kn.rowptr, kn.colidx, kn.w, np.arange(n), np.full(n, 1 / n)) != \
        pytest.approx(want, rel=1e-6)
    monkeypatch.setattr(dense, "effective_resistance", lambda *a: orig(*a) ** 2)
    assert dense.network_variance(kn.n, kn.rowptr, kn.colidx, kn.w, np.arange(n), np.full(n, 1 / n)) != \
        pytest.approx(want, rel=1e-6)


def test_effective_resistance_pin_catches_sign_mistake(monkeypatch):
    """A copy with L^+_uu + L^+_vv + 2 L^+_uv (wrong sign) fails the path pin."""
    orig = dense.pinv_laplacian
    monkeypatch.setattr(dense, "pinv_laplacian", lambda L, c: orig(L, c) * np.where(np.eye(len(L)) > 0, 1.0, -1.0))
    g = graph(6, *synth.path_graph(6))
    assert dense.effective_resistance(g.n, g.rowptr, g.colidx, g.w, [0], [5])[0] != pytest.approx(5.0, rel=1e-6)


def test_network_variance_closed_forms():
    """Variance of the uniform distribution is tr(L^+)/n (the sum of all effective
    resistances is 2n tr L^+), so with the textbook Laplacian spectra: K_n with
    weight w gives (n-1)/(n^2 w), the unit cycle C_n gives (n^2-1)/(12n).  A point
    mass has variance 0 and two equal masses have R/4."""
    n, wgt = 9, 1.7
    kn = graph(n, *synth.complete_graph(n), np.full(n * (n - 1) // 2, wgt))
    u = np.full(n, 1.0 / n)
    assert dense.network_variance(kn.n, kn.rowptr, kn.colidx, kn.w, np.arange(n), u) == \
        pytest.approx((n - 1) / (n * n * wgt), rel=1e-12)
    m = 11
    cyc = graph(m, *synth.cycle_graph(m))
    assert dense.network_variance(cyc.n, cyc.rowptr, cyc.colidx, cyc.w, np.arange(m), np.full(m, 1.0 / m)) == \
        pytest.approx((m * m - 1) / (12 * m), rel=1e-12)
    pth = graph(7, *synth.path_graph(7))
    assert dense.network_variance(pth.n, pth.rowptr, pth.colidx, pth.w, [3], [1.0]) == 0.0
    assert dense.network_variance(pth.n, pth.rowptr, pth.colidx, pth.w, [1, 6], [0.5, 0.5]) == \
        pytest.approx(5 / 4, rel=1e-12)
    two = synth.disjoint_union([pth, cyc])[0]
    assert dense.network_variance(two.n, two.rowptr, two.colidx, two.w, [0, 9], [0.5, 0.5]) == np.inf
    assert dense.network_variance(two.n, two.rowptr, two.colidx, two.w, [0, 9], [1.0, 0.0]) == 0.0


# ---------------------------------------------------------------- invariants

def _ba(n=60, seed=1, weighted=True):
    rng = np.random.default_rng(seed)
    eu, ev = synth.barabasi_albert(n, 2, rng)
    wts = rng.uniform(0.5, 2.0, size=len(eu)) if weighted else None
    return graph(n, eu, ev, wts)


@pytest.mark.parametrize("route", ROUTES)
def test_metric_axioms(route):
    g = _ba()
    rng = np.random.default_rng(2)
    V = rng.random((4, g.n))
    dd = np.zeros((4, 4))
    for a, b in itertools.product(range(4), range(4)):
        dd[a, b] = np.sqrt(max(d2(g, V[a], V[b], route)[0], 0.0))
    assert np.allclose(dd, dd.T, rtol=1e-11, atol=1e-13)
    assert np.all(np.abs(np.diag(dd)) < 1e-7)
    for a, b, c in itertools.permutations(range(4), 3):
        assert dd[a, c] <= dd[a, b] + dd[b, c] + 1e-12


@pytest.mark.parametrize("route", ROUTES)
def test_shift_scale_and_weight_scaling(route):
    g = _ba()
    rng = np.random.default_rng(4)
    x, y = rng.random(g.n), rng.random(g.n)
    base = d2(g, x, y, route)[0]
    assert d2(g, x + 3.7, y, route)[0] == pytest.approx(base, rel=1e-10)
    assert d2(g, -2.5 * x, -2.5 * y, route)[0] == pytest.approx(6.25 * base, rel=1e-10)
    g2 = synth.csr_from_edges(g.n, g.eu, g.ev, g.ew * 4.0)
    assert d2(g2, x, y, route)[0] == pytest.approx(base / 4.0, rel=1e-10)


@pytest.mark.parametrize("route", ROUTES)
def test_permutation_invariance(route):
    g = _ba()
    rng = np.random.default_rng(9)
    x, y = rng.random(g.n), rng.random(g.n)
    base = d2(g, x, y, route)[0]
    perm = rng.permutation(g.n)         # new label of old node i is perm[i]
    gp = synth.csr_from_edges(g.n, perm[g.eu], perm[g.ev], g.ew)
    xp = np.empty_like(x)
    yp = np.empty_like(y)
    xp[perm] = x
    yp[perm] = y
    assert d2(gp, xp, yp, route)[0] == pytest.approx(base, rel=1e-10)


@pytest.mark.parametrize("route", ROUTES)
def test_disconnected_projection(route):
    """Two components plus an isolated node: d^2 is the sum of per-component d^2 of the
    per-component mean-zero delta; constants per component and the isolated node drop out."""
    rng = np.random.default_rng(13)
    ga = _ba(30, seed=21)
    gb = _ba(25, seed=22)
    iso = graph(1, np.empty(0, np.int64), np.empty(0, np.int64))
    gu, offs = synth.disjoint_union([ga, iso, gb])
    x, y = rng.random(gu.n), rng.random(gu.n)
    parts = 0.0
    for gg, o in [(ga, offs[0]), (gb, offs[2])]:
        parts += d2(gg, x[o:o + gg.n], y[o:o + gg.n], "eig")[0]
    assert d2(gu, x, y, route)[0] == pytest.approx(parts, rel=1e-10)
    x2 = x.copy()
    x2[offs[2]:offs[2] + gb.n] += 5.0
    x2[offs[1]] += 9.0
    assert d2(gu, x2, y, route)[0] == pytest.approx(parts, rel=1e-10)


def test_selfloop_ignored_and_duplicates_summed():
    """L ignores self-loops and sums repeated entries (parallel conductances)."""
    base = _ba(20, seed=5)
    rng = np.random.default_rng(6)
    x, y = rng.random(base.n), rng.random(base.n)
    want = d2(base, x, y, "eig")[0]
    # split every stored weight into two repeated entries and add a self-loop on row 0
    rows = np.repeat(np.arange(base.n), np.diff(base.rowptr))
    r2 = np.concatenate([rows, rows, [0]])
    c2 = np.concatenate([base.colidx, base.colidx, [0]])
    w2 = np.concatenate([0.3 * base.w, 0.7 * base.w, [42.0]])
    order = np.lexsort((c2, r2))
    r2, c2, w2 = r2[order], c2[order], w2[order]
    rowptr = np.zeros(base.n + 1, dtype=np.int64)
    np.cumsum(np.bincount(r2, minlength=base.n), out=rowptr[1:])
    got = dense.ge_d2_eig(base.n, rowptr, c2, w2, x[None], y[None])[0]
    assert got == pytest.approx(want, rel=1e-11)
    got2 = dense.ge_d2_grounded(base.n, rowptr, c2, w2, x[None], y[None])[0]
    assert got2 == pytest.approx(want, rel=1e-11)


def test_asymmetric_storage_uses_symmetric_part():
    """Under the W_sym reading, scaling w_uv by (1+t) and w_vu by (1-t) changes nothing."""
    g = _ba(25, seed=8)
    pos_uv, pos_vu = g.edge_positions()
    w = g.w.copy()
    w[pos_uv[0]] *= 1.4
    w[pos_vu[0]] *= 0.6
    rng = np.random.default_rng(1)
    x, y = rng.random(g.n), rng.random(g.n)
    a = dense.ge_d2_eig(g.n, g.rowptr, g.colidx, g.w, x[None], y[None])[0]
    b = dense.ge_d2_eig(g.n, g.rowptr, g.colidx, w, x[None], y[None])[0]
    assert b == pytest.approx(a, rel=1e-12)


# ---------------------------------------------------------------- route agreement

def test_dense_routes_agree_on_workload_ba_small():
    wl = synth.workload_ba_small()
    g = wl.graph
    X, Y = wl.pairs(0, 16)
    a = dense.ge_d2_eig(g.n, g.rowptr, g.colidx, g.w, X, Y)
    b = dense.ge_d2_grounded(g.n, g.rowptr, g.colidx, g.w, X, Y)
    c, it, rr = cg.ge_d2_cg(g.n, g.rowptr, g.colidx, g.w, X, Y, rtol=1e-12)
    assert np.all(it > 0) and np.all(rr <= 1e-12)
    assert np.max(np.abs(a - b) / a) < 1e-12
    assert np.max(np.abs(a - c) / a) < 1e-10


def test_cg_thread_count_does_not_change_result_beyond_rounding():
    g = _ba(400, seed=31)
    rng = np.random.default_rng(0)
    X, Y = rng.random((3, g.n)), rng.random((3, g.n))
    a = cg.ge_d2_cg(g.n, g.rowptr, g.colidx, g.w, X, Y, threads=1)[0]
    b = cg.ge_d2_cg(g.n, g.rowptr, g.colidx, g.w, X, Y, threads=5)[0]
    assert np.allclose(a, b, rtol=1e-12)


def test_tiny_graphs_property():
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    @hyp.settings(max_examples=60, deadline=None)
    @hyp.given(n=st.integers(2, 12), p=st.floats(0.1, 0.9), seed=st.integers(0, 10**6))
    def check(n, p, seed):
        rng = np.random.default_rng(seed)
        eu, ev = synth.random_gnp_small(n, p, rng)
        wts = rng.uniform(0.1, 5.0, size=len(eu))
        g = graph(n, eu, ev, wts)
        X, Y = rng.random((2, n)), rng.random((2, n))
        a = d2(g, X, Y, "eig")
        b = d2(g, X, Y, "grounded")
        c = d2(g, X, Y, "cg")
        scale = max(1e-300, np.max(np.abs(a)))
        assert np.max(np.abs(a - b)) <= 1e-10 * scale
        assert np.max(np.abs(a - c)) <= 1e-9 * scale
        assert np.all(a >= -1e-12 * scale)

    check()


# ---------------------------------------------------------------- gradients

def test_gradient_matches_central_differences():
    """d(d^2)/dx = 2 z and d(d^2)/dW_uv = -1/2 (z_u - z_v)^2 per stored entry, against
    FP64 central differences (h = 1e-6)."""
    g = _ba(30, seed=17)
    rng = np.random.default_rng(17)
    X, Y = rng.random((2, g.n)), rng.random((2, g.n))
    gbar = np.array([0.7, -1.3])
    gw, gx, gy = dense.ge_grad_dense(g.n, g.rowptr, g.colidx, g.w, X, Y, gbar)

    def f(w=None, X_=None, Y_=None):
        return float(gbar @ dense.ge_d2_eig(g.n, g.rowptr, g.colidx,
                                            g.w if w is None else w,
                                            X if X_ is None else X_, Y if Y_ is None else Y_))

    h = 1e-6
    # central differences of an O(1) FP64 function at h = 1e-6 carry ~1e-10/h absolute noise
    tol = 1e-7 * max(1.0, abs(f()))
    for e in rng.choice(g.nnz, size=8, replace=False):
        wp = g.w.copy(); wp[e] += h
        wm = g.w.copy(); wm[e] -= h
        fd = (f(w=wp) - f(w=wm)) / (2 * h)
        assert fd == pytest.approx(gw[e], rel=1e-5, abs=tol)
    for (p, i) in [(0, 3), (1, 17), (0, 29)]:
        Xp = X.copy(); Xp[p, i] += h
        Xm = X.copy(); Xm[p, i] -= h
        fd = (f(X_=Xp) - f(X_=Xm)) / (2 * h)
        assert fd == pytest.approx(gx[p, i], rel=1e-5, abs=tol)
        Yp = Y.copy(); Yp[p, i] += h
        Ym = Y.copy(); Ym[p, i] -= h
        fd = (f(Y_=Yp) - f(Y_=Ym)) / (2 * h)
        assert fd == pytest.approx(gy[p, i], rel=1e-5, abs=tol)


def test_gradient_path_closed_form():
    """On a weighted path R_{0,n-1} = sum 1/w_e, so dR/dw_e = -1/w_e^2 per undirected edge
    (the two stored entries of an edge together)."""
    n = 12
    rng = np.random.default_rng(23)
    wts = rng.uniform(0.5, 2.0, size=n - 1)
    g = graph(n, *synth.path_graph(n), wts)
    x = np.zeros(n); y = np.zeros(n)
    x[0] = 1.0; y[n - 1] = 1.0
    gw, _, _ = dense.ge_grad_dense(g.n, g.rowptr, g.colidx, g.w, x[None], y[None], [1.0])
    puv, pvu = g.edge_positions()
    per_edge = gw[puv] + gw[pvu]
    order = np.argsort(g.eu)
    assert np.allclose(per_edge[order], -1.0 / wts ** 2, rtol=1e-10)


# ---------------------------------------------------------------- planted mistakes

def test_pins_catch_planted_mistakes(monkeypatch):
    """Copies of the oracle with a plausible mistake must fail at least one pin."""
    star = graph(5, *synth.star_graph(4), np.array([0.5, 2.0, 4.0, 1.0]))
    want_star = 1 / 0.5 + 1 / 2.0
    orig_lap = dense.laplacian_dense

    # (1) dropped 1/2 of the W_sym split (every weight counted twice)
    def lap_double(n, rowptr, colidx, w):
        return 2.0 * orig_lap(n, rowptr, colidx, w)
    monkeypatch.setattr(dense, "laplacian_dense", lap_double)
    assert resistance(star, 1, 2, "eig") != pytest.approx(want_star, rel=1e-6)
    monkeypatch.setattr(dense, "laplacian_dense", orig_lap)

    # (2) wrong sign on the off-diagonal (D + W instead of D - W)
    def lap_signless(n, rowptr, colidx, w):
        L = orig_lap(n, rowptr, colidx, w)
        return np.abs(L)
    monkeypatch.setattr(dense, "laplacian_dense", lap_signless)
    # (a bipartite graph hides this mistake: there D + W is similar to D - W, so the
    # non-bipartite complete-graph pin is the one that must catch it)
    kn = graph(7, *synth.complete_graph(7))
    assert resistance(kn, 0, 5, "grounded") != pytest.approx(2.0 / 7, rel=1e-6)
    monkeypatch.setattr(dense, "laplacian_dense", orig_lap)

    # (3) one zero eigenvalue too few dropped on a disconnected graph: caught by the
    # per-component pin with vectors whose component means differ
    pa, pb = graph(4, *synth.path_graph(4)), graph(3, *synth.path_graph(3))
    two = synth.disjoint_union([pa, pb])[0]
    rng = np.random.default_rng(0)
    x, y = rng.random(7), rng.random(7)
    want = d2(pa, x[:4], y[:4], "eig")[0] + d2(pb, x[4:], y[4:], "eig")[0]
    orig_pinv = dense.pinv_laplacian
    monkeypatch.setattr(dense, "pinv_laplacian", lambda L, c: orig_pinv(L, max(c - 1, 1)))
    with np.errstate(all="ignore"):
        got = d2(two, x, y, "eig")[0]
    assert not (abs(got - want) < 1e-6 * abs(want))
    monkeypatch.setattr(dense, "pinv_laplacian", orig_pinv)

    # (4) transposed pair of operands in the gradient (z_u - z_u): path closed form fails
    n = 5
    gpath = graph(n, *synth.path_graph(n), np.array([1.0, 2.0, 0.5, 1.5]))
    x = np.zeros(n); y = np.zeros(n); x[0] = 1; y[-1] = 1
    Z = dense.ge_z_dense(gpath.n, gpath.rowptr, gpath.colidx, gpath.w, x[None], y[None])
    rows = np.repeat(np.arange(n), np.diff(gpath.rowptr))
    wrong = -0.5 * (Z[0, rows] - Z[0, rows]) ** 2
    puv, pvu = gpath.edge_positions()
    assert not np.allclose((wrong[puv] + wrong[pvu]), -1.0 / gpath.ew ** 2)
