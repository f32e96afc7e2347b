"""Warm start (nvd_ge_distance_warm): the solve starts from a saved z0 instead of
z = 0.  It must reach the oracle's d^2 (variational estimate, FP64 tolerance 1e-8)
from any start, ignore constants per component in z0, stop at once when z0 is
already the solution, and need fewer iterations when z0 is close (the weights
changed a little, as between steps of a gradient-based fit)."""
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


@pytest.fixture(scope="module")
def ba():
    wl = synth.workload_ba_small()
    g0 = wl.graph
    rng = np.random.default_rng(12)
    g = synth.csr_from_edges(g0.n, g0.eu, g0.ev, rng.uniform(0.5, 2.0, g0.m))
    X, Y = wl.pairs(0, 16)
    want = dense.ge_d2_eig(g.n, g.rowptr, g.colidx, g.w, X, Y)
    return g, X, Y, want


@pytest.mark.parametrize("kw", [dict(single_rhs=True), dict(kt=8), dict(kt=8, fold_direction=True)])
def test_warm_from_its_own_solution(nvd, ba, kw):
    g, X, Y, want = ba
    G = nvd.Graph.from_csr(g)
    d2, z, st = nvd.ge_distance(G, on(X), on(Y), rtol=1e-11, return_z=True, return_stats=True, **kw)
    d2w, zw, stw = nvd.ge_distance(G, on(X), on(Y), rtol=1e-11, z0=z, return_z=True, return_stats=True, **kw)
    assert rel(d2w.cpu().numpy(), want) < 1e-8
    assert rel(d2w.cpu().numpy(), d2.cpu().numpy()) < 1e-10
    assert all(s["iters"] <= 3 and s["status"] == 0 for s in stw)
    assert all(s["rel_resid"] <= 1e-10 for s in stw)          # the true residual at the end
    assert torch.max(torch.abs(zw - z)).item() <= 1e-7 * torch.max(torch.abs(z)).item()
    # z0 may be the output buffer itself
    d2s = nvd.ge_distance(G, on(X), on(Y), rtol=1e-11, z0=zw, **kw)
    assert rel(d2s.cpu().numpy(), want) < 1e-8


def test_warm_zero_start_equals_cold(nvd, ba):
    g, X, Y, want = ba
    G = nvd.Graph.from_csr(g)
    d2c, stc = nvd.ge_distance(G, on(X), on(Y), rtol=1e-11, return_stats=True)
    d2w, stw = nvd.ge_distance(G, on(X), on(Y), rtol=1e-11, z0=torch.zeros_like(on(X)), return_stats=True)
    assert rel(d2w.cpu().numpy(), d2c.cpu().numpy()) < 1e-10
    assert all(abs(a["iters"] - b["iters"]) <= 1 for a, b in zip(stw, stc))


def test_warm_after_weight_change(nvd):
    """ER n = 20,000, mean degree 8: solve, change every weight by up to 1%, solve
    again cold and warm from the old z; both match the oracle on the new weights
    and the warm solve takes fewer iterations."""
    rng = np.random.default_rng(21)
    g0 = synth.sweep_graph("er", 20000, 8, seed=3)
    w = rng.uniform(0.5, 2.0, g0.m)
    g1 = synth.csr_from_edges(g0.n, g0.eu, g0.ev, w)
    g2 = synth.csr_from_edges(g0.n, g0.eu, g0.ev, w * (1.0 + 0.01 * rng.uniform(-1, 1, g0.m)))
    X, Y = synth.sparse_uniform_pairs(g0.n, 8, 0.10, 9)
    want, it, _ = ocg.ge_d2_cg(g2.n, g2.rowptr, g2.colidx, g2.w, X, Y, rtol=1e-13)
    assert np.all(it > 0)
    _, z1 = nvd.ge_distance(nvd.Graph.from_csr(g1), on(X), on(Y), rtol=1e-10, return_z=True, kt=8)
    G2 = nvd.Graph.from_csr(g2)
    d2c, stc = nvd.ge_distance(G2, on(X), on(Y), rtol=1e-10, return_stats=True, kt=8)
    d2w, stw = nvd.ge_distance(G2, on(X), on(Y), rtol=1e-10, z0=z1, return_stats=True, kt=8)
    assert rel(d2c.cpu().numpy(), want) < 1e-8
    assert rel(d2w.cpu().numpy(), want) < 1e-8
    assert all(s["status"] == 0 and s["rel_resid"] <= 1e-9 for s in stw)
    assert sum(s["iters"] for s in stw) < sum(s["iters"] for s in stc)


@pytest.mark.parametrize("kt", [1, 8])
def test_warm_disconnected_with_null_space_start(nvd, kt):
    """Components interleaved in the user's order plus isolated nodes (relabelling
    path), 13 pairs (ragged last tile): z0 = the dense oracle's z plus a different
    constant on every component plus noise of relative size 1e-3.  d^2 and z_out
    (mean-zero per component) match the oracle."""
    rng = np.random.default_rng(5)
    parts = []
    for n_i in (120, 80, 60):
        eu, ev = synth.barabasi_albert(n_i, 2, rng)
        parts.append(synth.csr_from_edges(n_i, eu, ev, rng.uniform(0.5, 2.0, len(eu))))
    u0, _ = synth.disjoint_union(parts)
    n = u0.n + 4
    lab = rng.permutation(n)
    g = synth.csr_from_edges(n, lab[u0.eu], lab[u0.ev], u0.ew)
    X, Y = rng.random((13, n)), rng.random((13, n))
    want = dense.ge_d2_eig(g.n, g.rowptr, g.colidx, g.w, X, Y)
    zref = dense.ge_z_dense(g.n, g.rowptr, g.colidx, g.w, X, Y)
    comp, c = dense.components(g.n, g.rowptr, g.colidx)
    shift = rng.normal(0, 5.0, c)[comp]
    z0 = zref + shift[None, :] + 1e-3 * np.abs(zref).max() * rng.standard_normal(zref.shape)
    G = nvd.Graph.from_csr(g)
    d2, z, st = nvd.ge_distance(G, on(X), on(Y), rtol=1e-12, kt=kt, z0=on(z0), return_z=True, return_stats=True)
    assert rel(d2.cpu().numpy(), want) < 1e-8
    zz = z.cpu().numpy()
    iso = np.bincount(comp)[comp] == 1
    assert np.all(zz[:, iso] == 0.0)
    assert np.max(np.abs(zz - zref)) <= 1e-7 * np.max(np.abs(zref))
    assert all(s["status"] == 0 for s in st)


def test_warm_invalid_uses(nvd, ba):
    g, X, Y, _ = ba
    G = nvd.Graph.from_csr(g)
    z0 = torch.zeros_like(on(X))
    for mode in (nvd.MODE_FP32, nvd.MODE_MIXED):
        with pytest.raises(nvd.NvdError) as e:
            nvd.ge_distance(G, on(X), on(Y), mode=mode, z0=z0)
        assert e.value.status == 1
    with pytest.raises(ValueError):
        nvd.ge_distance(G, X, Y, z0=z0)                      # host inputs
    with pytest.raises(ValueError):
        nvd.ge_distance(G, on(X), on(Y), z0=z0[:3])
