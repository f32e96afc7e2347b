"""The allocation-free entry point nvd_laplacian_quadform_noalloc (for callers that
cannot allocate device memory when they call: its partial sums live in a fixed
device array inside the library instead of handle workspace).

Called through the C ABI twice in a row and compared with the existing entry
point nvd_laplacian_apply (y = L x), with x^T y from that output and with the
oracle's dense Laplacian (y = L x, q = x^T L x in FP64 on the host).  A larger
graph reaches the launch's block cap (every partial-sum slot in use) with the
maximum of 32 columns and no y.  This file is collected last so a run that stops
at the first failure has run every other test first.
"""
import ctypes

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
    lib = m.load_library()
    fn = lib.nvd_laplacian_quadform_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p]
    return m


def graphs():
    rng = np.random.default_rng(3)
    base = synth.workload_grad(0.002).graph                          # BA m=5, FP32 weights
    parts = []
    for seed, n in [(1, 300), (2, 1), (3, 200)]:
        r = np.random.default_rng(seed)
        if n == 1:
            parts.append(synth.csr_from_edges(1, np.empty(0, np.int64), np.empty(0, np.int64), np.empty(0)))
        else:
            eu, ev = synth.barabasi_albert(n, 3, r)
            parts.append(synth.csr_from_edges(n, eu, ev, r.uniform(0.5, 2, size=len(eu))))
    gu, _ = synth.disjoint_union(parts)
    perm = rng.permutation(gu.n)                                      # interleaved components
    mixed = synth.csr_from_edges(gu.n, perm[gu.eu], perm[gu.ev], gu.ew)
    return [base, mixed]


@pytest.mark.parametrize("gi", [0, 1])
def test_noalloc_matches_existing_entry_point_twice(nvd, gi):
    g = graphs()[gi]
    G = nvd.Graph.from_csr(g)
    lib = nvd.load_library()
    rng = np.random.default_rng(10 + gi)
    k = 5
    X = torch.as_tensor(rng.standard_normal((k, g.n)), device=DEV)
    y_ref = nvd.laplacian_apply(G, X)                                  # existing entry point
    q_ref = (X * y_ref).sum(dim=1)
    scale = float(y_ref.abs().max())
    for _ in range(2):                                                 # two calls in a row
        y = torch.full_like(X, float("nan"))
        q = torch.full((k,), float("nan"), dtype=torch.float64, device=DEV)
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = lib.nvd_laplacian_quadform_noalloc(G.handle, k, X.data_ptr(), y.data_ptr(), q.data_ptr(), stream)
        assert rc == 0, lib.nvd_last_error()
        torch.cuda.synchronize()
        assert float((y - y_ref).abs().max()) <= 1e-12 * scale
        assert torch.allclose(q, q_ref, rtol=1e-10, atol=1e-12 * float(q_ref.abs().max()))
    # the oracle's dense L (FP64, host): y = L x and q = x^T L x column by column
    L = dense.laplacian_dense(g.n, g.rowptr, g.colidx, g.w.astype(np.float64))
    Xh = X.cpu().numpy()
    y_or = Xh @ L                                                      # L is symmetric
    q_or = np.einsum("kn,kn->k", Xh, y_or)
    assert np.max(np.abs(y.cpu().numpy() - y_or)) <= 1e-12 * np.max(np.abs(y_or))
    assert np.max(np.abs(q.cpu().numpy() - q_or) / np.abs(q_or)) <= 1e-10


def test_noalloc_at_the_block_cap_with_32_columns_and_no_y(nvd):
    """n = 50,000 (BA m = 4): the launch is capped (1024 blocks, or 8 per SM), every
    one of the 32 partial-sum columns is in use and y is NULL; q against x^T (L x)
    of the existing entry point, twice in a row."""
    r = np.random.default_rng(41)
    eu, ev = synth.barabasi_albert(50_000, 4, r)
    g = synth.csr_from_edges(50_000, eu, ev, r.uniform(0.5, 2.0, size=len(eu)))
    G = nvd.Graph.from_csr(g)
    lib = nvd.load_library()
    k = 32
    X = torch.as_tensor(r.standard_normal((k, g.n)), device=DEV)
    q_ref = (X * nvd.laplacian_apply(G, X)).sum(dim=1)
    for _ in range(2):
        q = torch.full((k,), float("nan"), dtype=torch.float64, device=DEV)
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = lib.nvd_laplacian_quadform_noalloc(G.handle, k, X.data_ptr(), None, q.data_ptr(), stream)
        assert rc == 0, lib.nvd_last_error()
        torch.cuda.synchronize()
        assert torch.allclose(q, q_ref, rtol=1e-10, atol=0.0)


def test_noalloc_rejects_too_many_columns(nvd):
    g = graphs()[0]
    G = nvd.Graph.from_csr(g)
    lib = nvd.load_library()
    X = torch.zeros((33, g.n), dtype=torch.float64, device=DEV)
    q = torch.zeros(33, dtype=torch.float64, device=DEV)
    rc = lib.nvd_laplacian_quadform_noalloc(G.handle, 33, X.data_ptr(), None, q.data_ptr(), None)
    assert rc == 1
    assert b"maximum of 32" in lib.nvd_last_error()
