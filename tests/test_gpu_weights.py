"""New weights on an existing handle (nvd_graph_set_weights): the weighted graphs of
Section 3.1 with w changing between evaluations, as in a training loop that
differentiates d^2 with respect to w.  After the update every solve mode, cached
tile plan, batched union and the autograd path must see the new weights (oracle
parity on the new weights, no graph rebuild), the mapping of the caller's entries
(repeats, self-loops, relabelled components) must equal a fresh creation, and a
rejected update must leave the handle as it was."""
import ctypes

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


def on(a, dtype=torch.float64):
    return torch.as_tensor(a, dtype=dtype, device=DEV)


def test_optimizer_step_on_w_then_d2_and_grad_on_the_new_weights(nvd):
    """Gradient steps on w (FP32, requires_grad, updated in place) through the autograd
    path on one handle: after each step d^2 and the gradients match the dense oracle
    on the updated weights."""
    wl = synth.workload_grad(0.002)                         # BA n = 2,000, m = 5, lognormal FP32
    g = wl.graph
    X, Y = wl.pairs(0, 6)
    G = nvd.Graph.from_csr(g)
    w = torch.as_tensor(g.w, device=DEV).clone().requires_grad_(True)
    x = on(X).requires_grad_(True)
    y = on(Y)
    gbar = np.random.default_rng(3).uniform(0.5, 1.5, 6)
    for step in range(3):
        w.grad = None
        x.grad = None
        d2 = nvd.ge_distance_autograd(G, x, y, w, rtol=1e-12)
        (d2 * on(gbar)).sum().backward()
        w_now = w.detach().cpu().numpy().astype(np.float64)
        want = dense.ge_d2_eig(g.n, g.rowptr, g.colidx, w_now, X, Y)
        assert rel(d2.detach().cpu().numpy(), want) < 1e-9, step
        gw_ref, gx_ref, _ = dense.ge_grad_dense(g.n, g.rowptr, g.colidx, w_now, X, Y, gbar)
        assert np.max(np.abs(w.grad.cpu().numpy() - gw_ref)) <= 1e-6 * np.max(np.abs(gw_ref))
        assert np.max(np.abs(x.grad.cpu().numpy() - gx_ref)) <= 1e-8 * np.max(np.abs(gx_ref))
        with torch.no_grad():                               # a normalised gradient step, in place
            w -= 0.3 * w.grad / w.grad.abs().max()          # (bumps w's version)
            w.clamp_(min=1e-3)
    assert not np.allclose(w.detach().cpu().numpy(), g.w)  # the weights did move


def messy_csr(rng):
    """Two BA components interleaved by a node permutation, an isolated node, a
    self-loop on every 7th node and every 5th edge stored twice (both directions):
    creation drops, merges and relabels."""
    a_u, a_v = synth.barabasi_albert(150, 3, rng)
    b_u, b_v = synth.barabasi_albert(120, 2, rng)
    eu = np.concatenate([a_u, b_u + 150])
    ev = np.concatenate([a_v, b_v + 150])
    n = 271
    lab = rng.permutation(n)
    eu, ev = lab[eu], lab[ev]
    rows, cols, idx = [], [], []
    for k, (u, v) in enumerate(zip(eu, ev)):
        rep = 2 if k % 5 == 0 else 1
        for _ in range(rep):
            rows += [u, v]
            cols += [v, u]
            idx += [k, k]
    loops = np.arange(0, n, 7)
    rows += list(loops)
    cols += list(loops)
    idx += [-1] * len(loops)
    rows, cols, idx = np.array(rows), np.array(cols), np.array(idx)
    order = np.lexsort((cols, rows))
    rows, cols, idx = rows[order], cols[order], idx[order]
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)

    def weights(seed):
        r = np.random.default_rng(seed)
        we = r.uniform(0.5, 2.0, len(eu))
        # a repeated edge's two stored copies each carry half of its conductance
        reps = np.bincount(idx[idx >= 0], minlength=len(eu)) / 2
        out = np.where(idx >= 0, we[np.maximum(idx, 0)] / reps[np.maximum(idx, 0)], 1.0 + r.random(len(idx)))
        return out

    return n, rowptr, cols.astype(np.int32), weights


def test_entry_mapping_equals_a_fresh_creation(nvd):
    """Repeated entries, self-loops and relabelled components: a handle updated with new
    weights gives bitwise the d^2 and z of a handle created from them, in FP64, FP32
    and MIXED, and the weight gradient lands on the caller's entries."""
    rng = np.random.default_rng(11)
    n, rowptr, colidx, weights = messy_csr(rng)
    w0, w1 = weights(1), weights(2)
    X, Y = rng.random((5, n)), rng.random((5, n))
    G = nvd.Graph(rowptr, colidx, w0)
    assert G.info()["ncomp"] == 3
    for mode, kw in ((0, dict(rtol=1e-12)), (1, dict(rtol=1e-6)), (2, dict(rtol=1e-4, d2_rtol=1e-12))):
        nvd.ge_distance(G, on(X), on(Y), mode=mode, kt=4, **kw)     # build plans and the FP32 copy first
    G.set_weights(w1)
    F = nvd.Graph(rowptr, colidx, w1)
    for mode, kw in ((0, dict(rtol=1e-12)), (1, dict(rtol=1e-6)), (2, dict(rtol=1e-4, d2_rtol=1e-12))):
        a, za = nvd.ge_distance(G, on(X), on(Y), mode=mode, kt=4, return_z=True, **kw)
        b, zb = nvd.ge_distance(F, on(X), on(Y), mode=mode, kt=4, return_z=True, **kw)
        assert torch.equal(a, b), mode
        assert torch.equal(za, zb), mode
    # against the oracle on the new weights (its own cleaning of the same CSR)
    want = dense.ge_d2_eig(n, rowptr, colidx, w1, X, Y)
    d2, z = nvd.ge_distance(G, on(X), on(Y), rtol=1e-12, return_z=True)
    assert rel(d2.cpu().numpy(), want) < 1e-9
    gw, _, _ = nvd.ge_grad(G, z, on(np.ones(5)))
    gwf, _, _ = nvd.ge_grad(F, z, on(np.ones(5)))
    assert torch.equal(gw, gwf)


def test_rejected_updates_leave_the_handle_unchanged(nvd):
    rng = np.random.default_rng(5)
    wl = synth.workload_ba_small(0.2)
    g = wl.graph
    w = rng.uniform(0.5, 2.0, g.m)
    gw = synth.csr_from_edges(g.n, g.eu, g.ev, w)
    X, Y = wl.pairs(0, 4)
    G = nvd.Graph.from_csr(gw)
    before = nvd.ge_distance(G, on(X), on(Y), rtol=1e-12)
    bad = gw.w.copy()
    bad[7] = -1.0
    with pytest.raises(nvd.NvdError) as e:
        G.set_weights(bad)
    assert e.value.status == 3                                    # NVD_ERR_BAD_WEIGHT
    bad = gw.w.copy()
    bad[3] = np.nan
    with pytest.raises(nvd.NvdError) as e:
        G.set_weights(on(bad))                                    # device pointer path
    assert e.value.status == 3
    asym = gw.w.copy()
    asym[0] *= 1.5                                                # w_uv != w_vu
    with pytest.raises(nvd.NvdError) as e:
        G.set_weights(asym)
    assert e.value.status == 2                                    # NVD_ERR_NOT_SYMMETRIC
    with pytest.raises(ValueError):
        G.set_weights(gw.w[:-1])
    lib = nvd.load_library()
    wf = np.ascontiguousarray(gw.w, np.float32)
    assert lib.nvd_graph_set_weights(G.handle, wf.ctypes.data, nvd.F32, 0, None) == 1   # other dtype
    after = nvd.ge_distance(G, on(X), on(Y), rtol=1e-12)
    assert torch.equal(before, after)


def test_batched_and_elimination_see_the_new_weights(nvd):
    """A batch built before the update is rebuilt (its union copied the old weights);
    the elimination is dropped with the old weights and redone on request."""
    rng = np.random.default_rng(8)
    graphs = [synth.workloads.batched_graph(gi, scale=0.02) for gi in (1, 2, 33)]
    pairs = [synth.workloads.batched_pairs(gr, gi) for gr, gi in zip(graphs, (1, 2, 33))]
    G = [nvd.Graph.from_csr(gr) for gr in graphs]
    xs = [on(Xp) for Xp, _ in pairs]
    ys = [on(Yp) for _, Yp in pairs]
    nvd.ge_distance_batched(G, xs, ys, mode=0, rtol=1e-11)
    w_new = rng.uniform(0.5, 2.0, graphs[1].m)
    g1 = synth.csr_from_edges(graphs[1].n, graphs[1].eu, graphs[1].ev, w_new.astype(np.float32))
    G[1].set_weights(g1.w)
    d2 = nvd.ge_distance_batched(G, xs, ys, mode=0, rtol=1e-11).numpy()
    for i, gr in enumerate([graphs[0], g1, graphs[2]]):
        want, it, _ = ocg.ge_d2_cg(gr.n, gr.rowptr, gr.colidx, gr.w.astype(np.float64), pairs[i][0], pairs[i][1],
                                   rtol=1e-12)
        assert rel(d2[32 * i:32 * i + 32], want) < 1e-8, i
    # elimination on a sparse graph: dropped by the update, redone on request
    sg = synth.sweep_graph("er", 3000, 3, seed=5)
    sg = synth.csr_from_edges(sg.n, sg.eu, sg.ev, rng.uniform(0.5, 2.0, sg.m))
    S = nvd.Graph.from_csr(sg)
    S.eliminate()
    Xs, Ys = synth.sparse_uniform_pairs(sg.n, 4, 0.1, 9)
    w2 = rng.uniform(0.5, 2.0, sg.m)
    s2 = synth.csr_from_edges(sg.n, sg.eu, sg.ev, w2)
    S.set_weights(s2.w)
    with pytest.raises(nvd.NvdError) as e:
        nvd.ge_distance(S, on(Xs), on(Ys), eliminate=True)
    assert e.value.status == 1
    S.eliminate()
    want = dense.ge_d2_eig(s2.n, s2.rowptr, s2.colidx, s2.w, Xs, Ys)
    got = nvd.ge_distance(S, on(Xs), on(Ys), rtol=1e-12, eliminate=True).cpu().numpy()
    assert rel(got, want) < 1e-9
