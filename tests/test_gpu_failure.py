"""Failure detection on the GPU without a fault: the persistent kernel's grid barrier
is a bounded wait (2 s); a diagnostic flag makes it wait for one arrival more than the
grid has, so every wait runs out.  The call must return NVD_ERR_TIMEOUT, and the
handle and the CUDA context must stay usable: the next call gives the oracle's d^2."""
import time

import numpy as np
import pytest

import synth
from oracle import dense

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def nvd():
    import paper_2310_11222_gb300 as m
    m.load_library()
    return m


def test_grid_barrier_timeout_is_reported_and_context_survives(nvd):
    wl = synth.workload_ba_small()
    g = wl.graph
    X, Y = wl.pairs(0, 4)
    want = dense.ge_d2_eig(g.n, g.rowptr, g.colidx, g.w, X, Y)
    G = nvd.Graph.from_csr(g)
    x = torch.as_tensor(X, device=DEV)
    y = torch.as_tensor(Y, device=DEV)
    t0 = time.perf_counter()
    with pytest.raises(nvd.NvdError) as e:
        nvd.ge_distance(G, x, y, rtol=1e-10, persistent=True, test_timeout=True)
    dt = time.perf_counter() - t0
    assert e.value.status == 8                      # NVD_ERR_TIMEOUT
    assert 1.5 < dt < 30.0                          # the bounded wait ran out, once per call
    torch.cuda.synchronize()                        # context still usable
    d2 = nvd.ge_distance(G, x, y, rtol=1e-10, persistent=True).cpu().numpy()
    assert np.max(np.abs(d2 - want) / want) < 1e-8
    d2 = nvd.ge_distance(G, x, y, rtol=1e-10).cpu().numpy()
    assert np.max(np.abs(d2 - want) / want) < 1e-8


def test_not_converged_and_numeric_statuses(nvd):
    """max_iter too small: NVD_ERR_NOT_CONVERGED per pair, results still written; a
    non-finite input: NVD_ERR_NUMERIC for that pair only."""
    wl = synth.workload_ba_small()
    g = wl.graph
    X, Y = wl.pairs(0, 4)
    G = nvd.Graph.from_csr(g)
    d2, st = nvd.ge_distance(G, torch.as_tensor(X, device=DEV), torch.as_tensor(Y, device=DEV), rtol=1e-10,
                             max_iter=3, return_stats=True, allow_not_converged=True)
    assert all(s["status"] == 6 and s["iters"] == 3 for s in st)
    assert np.all(np.isfinite(d2.cpu().numpy()))
    Xn = X.copy()
    Xn[2, 5] = np.nan
    with pytest.raises(nvd.NvdError) as e:
        nvd.ge_distance(G, torch.as_tensor(Xn, device=DEV), torch.as_tensor(Y, device=DEV), rtol=1e-10, kt=4)
    assert e.value.status == 7                      # NVD_ERR_NUMERIC
