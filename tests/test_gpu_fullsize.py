"""Full-size parity of the precision and differentiation workloads, through the C ABI,
on outputs the oracle computes one by one (sampled pairs, sampled edges) and on
properties that hold at any size.

* Power-law configuration model, n = 1e7 (gamma 2.3 on [2, 1e4], largest component,
  lognormal(0,1) FP32 weights), 128 pairs with 0.1% support: FP32 block-PCG inside
  FP64 refinement (the mixed mode at its default tile width) must match the C FP64
  CG oracle to relative error 1e-8 on eight seeded sample pairs (two in each tile
  of 32 columns).
* Barabasi-Albert n = 1e6, m = 5, lognormal(0,0.5) FP32 weights, 64 pairs with 10%
  support: forward d^2 and backward through the adjoint kernel (autograd).
  d^2 and grad_x = 2 z against the oracle for all pairs, grad_w on sampled entries
  against the oracle's z; the single-pair edge gradient against central finite
  differences (h = 1e-6) of the oracle's d^2; and the dense L^+ gradient on the
  induced 500-node subgraph of a BFS from a seeded node.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import breadth_first_order

import synth
from oracle import cg as ocg
from oracle import dense

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]
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


def test_powerlaw_full_size_mixed(nvd):
    wl = synth.workload_powerlaw()
    g = wl.graph
    assert g.n > 9_000_000 and np.diff(g.rowptr).max() > 1000
    X, Y = wl.pairs(0, 128)
    G = nvd.Graph.from_csr(g)
    xt = torch.as_tensor(X, device=DEV)
    yt = torch.as_tensor(Y, device=DEV)
    d2, st = nvd.ge_distance(G, xt, yt, mode=nvd.MODE_MIXED, rtol=1e-4, d2_rtol=1e-8, return_stats=True)
    d2 = d2.cpu().numpy()
    assert np.all(np.isfinite(d2)) and np.all(d2 > 0)
    assert all(s["status"] == 0 for s in st)
    rng = np.random.default_rng(5)
    pick = np.concatenate([32 * t + rng.choice(32, 2, replace=False) for t in range(4)])
    want, it, _ = ocg.ge_d2_cg(g.n, g.rowptr, g.colidx, g.w.astype(np.float64), X[pick], Y[pick], rtol=1e-12)
    assert np.all(it > 0)
    assert rel(d2[pick], want) < 1e-8


@pytest.fixture(scope="module")
def grad_case(nvd):
    wl = synth.workload_grad()
    g = wl.graph
    X, Y = wl.pairs(0, 64)
    G = nvd.Graph.from_csr(g)
    w = torch.as_tensor(g.w, device=DEV).requires_grad_(True)       # FP32, as the graph was built
    x = torch.as_tensor(X, device=DEV).requires_grad_(True)
    y = torch.as_tensor(Y, device=DEV)
    d2 = nvd.ge_distance_autograd(G, x, y, w, rtol=1e-11)
    gbar = torch.as_tensor(np.random.default_rng(9).uniform(0.5, 1.5, 64), device=DEV)
    (d2 * gbar).sum().backward()
    return g, X, Y, d2.detach().cpu().numpy(), w.grad.cpu().numpy(), x.grad.cpu().numpy(), gbar.cpu().numpy()


def test_grad_full_size_against_oracle_z(grad_case):
    """d^2, grad_x = 2 gbar z (all 64 pairs) and grad_w = -1/2 sum_p gbar_p (z_pu - z_pv)^2
    on 200 sampled stored entries, with z from the oracle's FP64 CG for every pair."""
    g, X, Y, d2, gw, gx, gbar = grad_case
    assert np.all(np.isfinite(gw)) and np.all(gw <= 0)
    want, it, _, Z = ocg.ge_d2_cg(g.n, g.rowptr, g.colidx, g.w.astype(np.float64), X, Y, rtol=1e-12,
                                  return_z=True)
    assert np.all(it > 0)
    assert rel(d2, want) < 1e-8
    ref = 2.0 * gbar[:, None] * Z                                    # oracle z is projected mean-zero
    assert np.max(np.abs(gx - ref)) <= 1e-7 * np.max(np.abs(ref))
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    es = np.random.default_rng(23).choice(len(g.colidx), 200, replace=False)
    diff = Z[:, rows[es]] - Z[:, g.colidx[es]]
    want_w = -0.5 * np.einsum("k,ke->e", gbar, diff * diff)
    assert np.max(np.abs(gw[es] - want_w)) <= 1e-6 * np.max(np.abs(want_w))


def test_grad_full_size_w_against_finite_differences(nvd):
    """One pair alone: the GPU edge gradient (both stored entries of the edge) on the
    three edges with the largest gradient among 10,000 sampled ones, against central
    differences (h = 1e-6) of the oracle's d^2 with both entries perturbed."""
    wl = synth.workload_grad()
    g = wl.graph
    X, Y = wl.pairs(5, 1)
    G = nvd.Graph.from_csr(g)
    w = torch.as_tensor(g.w, device=DEV).requires_grad_(True)
    d2 = nvd.ge_distance_autograd(G, torch.as_tensor(X, device=DEV), torch.as_tensor(Y, device=DEV), w,
                                  rtol=1e-12)
    d2.sum().backward()
    gw = w.grad.cpu().numpy().astype(np.float64)
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    cand = np.random.default_rng(17).choice(len(g.colidx), 10_000, replace=False)
    cand = cand[rows[cand] < g.colidx[cand]]
    top = cand[np.argsort(gw[cand])[:3]]                             # most negative
    w64 = g.w.astype(np.float64)
    h = 1e-6
    for e in top:
        u, v = rows[e], g.colidx[e]
        e2 = g.rowptr[v] + np.searchsorted(g.colidx[g.rowptr[v]:g.rowptr[v + 1]], u)
        assert g.colidx[e2] == u
        wp, wm = w64.copy(), w64.copy()
        wp[[e, e2]] += h
        wm[[e, e2]] -= h
        dp = ocg.ge_d2_cg(g.n, g.rowptr, g.colidx, wp, X, Y, rtol=1e-13)[0][0]
        dm = ocg.ge_d2_cg(g.n, g.rowptr, g.colidx, wm, X, Y, rtol=1e-13)[0][0]
        fd = (dp - dm) / (2 * h)
        assert abs((gw[e] + gw[e2]) - fd) <= 1e-4 * abs(fd), (e, gw[e] + gw[e2], fd)


def test_grad_induced_subgraph_against_dense(nvd):
    """The induced 500-node subgraph of a BFS from a seeded node of the n = 1e6 BA graph
    (connected by construction): gradients against the dense L^+ oracle."""
    wl = synth.workload_grad()
    g = wl.graph
    A = sp.csr_matrix((np.ones(len(g.colidx)), g.colidx, g.rowptr), shape=(g.n, g.n))
    start = int(np.random.default_rng(31).integers(g.n))
    order = breadth_first_order(A, start, directed=False, return_predecessors=False)[:500]
    keep = np.zeros(g.n, bool)
    keep[order] = True
    idx = -np.ones(g.n, np.int64)
    idx[order] = np.arange(500)
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    m = keep[rows] & keep[g.colidx] & (rows < g.colidx)
    sub = synth.csr_from_edges(500, idx[rows[m]], idx[g.colidx[m]], g.w[m])
    assert dense.components(sub.n, sub.rowptr, sub.colidx)[1] == 1
    rng = np.random.default_rng(37)
    X, Y = rng.random((8, 500)), rng.random((8, 500))
    gbar = rng.uniform(0.5, 1.5, 8)
    gw_ref, gx_ref, _ = dense.ge_grad_dense(sub.n, sub.rowptr, sub.colidx, sub.w.astype(np.float64), X, Y, gbar)
    G = nvd.Graph.from_csr(sub)
    w = torch.as_tensor(sub.w, device=DEV).requires_grad_(True)
    x = torch.as_tensor(X, device=DEV).requires_grad_(True)
    d2 = nvd.ge_distance_autograd(G, x, torch.as_tensor(Y, device=DEV), w, rtol=1e-12)
    (d2 * torch.as_tensor(gbar, device=DEV)).sum().backward()
    assert np.max(np.abs(w.grad.cpu().numpy() - gw_ref)) <= 1e-6 * np.max(np.abs(gw_ref))   # FP32 storage
    assert np.max(np.abs(x.grad.cpu().numpy() - gx_ref)) <= 1e-7 * np.max(np.abs(gx_ref))
