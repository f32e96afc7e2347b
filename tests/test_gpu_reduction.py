"""Cross-block sums in grouped form, and the FP32-mode inner product.  A pass with many partial-sum slots (blocks and
split heavy rows) adds them in two levels: groups of consecutive slots, then the
group sums (each in a fixed order).  A power-law graph of 4e5 nodes with hubs of
degree up to 1e4, cut into small blocks, makes every multi-column pass take that
path.  The host polls convergence every 8 iterations, so each tile also runs
passes after all of its columns stopped (its split rows are then skipped); the
next solves on the same handle must find every arrival counter back at zero:
repeated and interleaved solves give bitwise equal results and iteration counts,
and sampled pairs match the FP64 CG oracle."""
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


@pytest.fixture(scope="module")
def case():
    wl = synth.workload_powerlaw(scale=0.04)
    g = wl.graph
    assert g.n > 300_000 and np.diff(g.rowptr).max() > 2000
    X, Y = wl.pairs(0, 40)                     # 40 pairs: a ragged last tile at KT 16 and 32
    pick = np.array([0, 17, 33, 39])
    want = ocg.ge_d2_cg(g.n, g.rowptr, g.colidx, g.w.astype(np.float64), X[pick], Y[pick], rtol=1e-12)[0]
    return g, X, Y, pick, want


@pytest.mark.parametrize("mode,kt", [(0, 16), (1, 16), (1, 32), (2, 16), (2, 32)])
def test_grouped_sums_repeat_and_match_the_oracle(nvd, case, mode, kt):
    g, X, Y, pick, want = case
    kw = {0: dict(rtol=1e-11), 1: dict(rtol=1e-6), 2: dict(rtol=1e-5, d2_rtol=1e-10)}[mode]
    tol = {0: 1e-8, 1: 1e-4, 2: 1e-8}[mode]
    G = nvd.Graph.from_csr(g, reorder=True)
    G.set_tuning(mode=mode, kt=kt, blocks_pct=200)          # twice the default block count
    xt = torch.as_tensor(X, device=DEV)
    yt = torch.as_tensor(Y, device=DEV)

    def run(x, y):
        d2, st = nvd.ge_distance(G, x, y, mode=mode, kt=kt, check_every=8, return_stats=True, **kw)
        assert all(s["status"] == 0 for s in st)
        return d2, [s["iters"] for s in st]

    a, ia = run(xt, yt)
    assert rel(a.cpu().numpy()[pick], want) < tol
    b, ib = run(xt, yt)
    assert torch.equal(a, b) and ia == ib
    run(yt.flip(0), xt)                                      # another solve in between
    c, ic = run(xt, yt)
    assert torch.equal(a, c) and ia == ic


@pytest.mark.parametrize("n", [1, 1000, 1 << 20, 3_000_017])
def test_fp32_mode_inner_product_on_cancelling_vectors(nvd, n):
    """nvd_dot_f32 runs the reduction of the FP32-mode PCG (exact float products in
    double-float, FP64 block and cross-block sums).  Vectors whose terms cancel
    (pairs +-1e4 (1 + noise)) around a small remainder: its error stays below
    1e-12 * sum |a_i b_i| of the exact sum (math.fsum of the FP64 products, which
    are exact), where an FP32 accumulation misses by orders of magnitude more."""
    import math
    rng = np.random.default_rng(n)
    big = (1e4 * (1.0 + rng.random(n))).astype(np.float32)
    sign = np.where(np.arange(n) % 2 == 0, 1.0, -1.0).astype(np.float32)
    a = (sign * big + rng.normal(0.0, 1e-3, n)).astype(np.float32)
    b = (1.0 + 1e-3 * rng.random(n)).astype(np.float32)
    prod = a.astype(np.float64) * b.astype(np.float64)
    exact = math.fsum(prod.tolist())
    scale = float(np.sum(np.abs(prod)))
    got = nvd.dot_f32(torch.as_tensor(a, device=DEV), torch.as_tensor(b, device=DEV))
    assert abs(got - exact) <= 1e-12 * scale
    again = nvd.dot_f32(torch.as_tensor(a, device=DEV), torch.as_tensor(b, device=DEV))
    assert got == again                                        # fixed order: repeatable
    if n >= 1 << 20:
        naive = float(torch.sum(torch.as_tensor(a * b, device=DEV)).item())   # FP32 products and sums
        assert abs(naive - exact) > 1e3 * abs(got - exact)
