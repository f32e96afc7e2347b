"""Seeded random-graph generators returning symmetric CSR adjacency.

Every generator draws from a ``numpy.random.Generator`` passed in by the caller,
so a workload is reproducible from its seed alone.  The output is the
*adjacency* (off-diagonal weights) in CSR form with both directions of every
undirected edge stored, columns sorted within each row, no self-loops and no
duplicate entries.  Nothing here forms a Laplacian or any other quantity of the
method itself.

Graph models (Section 4.1.2 of the paper gives their outlines):

* Erdos-Renyi G(n, m): m distinct edges, endpoints uniform.
* Barabasi-Albert: growth from a star on m+1 nodes, each new node attaches to m
  distinct existing nodes chosen with probability proportional to degree.
* Watts-Strogatz: ring lattice with k nearest neighbours, the far end of every
  lattice edge rewired with probability p to a uniform node, avoiding
  self-loops and duplicate edges.
* Stochastic block model: groups with in-group probability p_in and
  out-group probability p_out.
* Erased configuration model with a discrete power-law degree sequence (the
  heavy-tailed workload): stubs paired uniformly, then self-loops and
  multi-edges erased.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csg


@dataclass
class CSRGraph:
    """Symmetric CSR adjacency of an undirected weighted graph.

    ``rowptr`` int64 [n+1], ``colidx`` int32 [nnz], ``w`` float32/float64 [nnz].
    ``eu, ev`` (int64, eu < ev) list every undirected edge once and ``ew`` its
    weight; ``epos_uv`` / ``epos_vu`` give the CSR positions of the two stored
    entries of each edge (used by per-edge gradient tests).
    """

    n: int
    rowptr: np.ndarray
    colidx: np.ndarray
    w: np.ndarray
    eu: np.ndarray = field(repr=False)
    ev: np.ndarray = field(repr=False)
    ew: np.ndarray = field(repr=False)
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    @property
    def m(self) -> int:
        return int(self.eu.shape[0])

    def edge_positions(self):
        """CSR positions (pos_uv, pos_vu) of the two stored entries of each edge."""
        def find(rows, cols):
            starts = self.rowptr[rows]
            ends = self.rowptr[rows + 1]
            out = np.empty(rows.shape[0], dtype=np.int64)
            # per-row sorted columns: vectorised binary search via a global key
            key = (np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.rowptr))
                   * self.n + self.colidx.astype(np.int64))
            q = rows.astype(np.int64) * self.n + cols.astype(np.int64)
            out[:] = np.searchsorted(key, q)
            assert np.all(out >= starts) and np.all(out < ends)
            return out
        return find(self.eu, self.ev), find(self.ev, self.eu)

    def structure_hash(self) -> str:
        """Short digest of (n, rowptr, colidx) to detect generator drift."""
        import hashlib
        h = hashlib.sha256()
        h.update(np.int64(self.n).tobytes())
        h.update(np.ascontiguousarray(self.rowptr, dtype=np.int64).tobytes())
        h.update(np.ascontiguousarray(self.colidx, dtype=np.int32).tobytes())
        return h.hexdigest()[:16]


def _canonical_unique(u: np.ndarray, v: np.ndarray, n: int):
    """Canonicalise (min, max), drop self-loops, keep first occurrence of each edge."""
    a = np.minimum(u, v).astype(np.int64)
    b = np.maximum(u, v).astype(np.int64)
    keep = a != b
    a, b = a[keep], b[keep]
    key = a * n + b
    _, first = np.unique(key, return_index=True)
    first.sort()
    return a[first], b[first]


def csr_from_edges(n: int, eu: np.ndarray, ev: np.ndarray, ew: np.ndarray,
                   name: str = "") -> CSRGraph:
    """Build symmetric CSR (both directions stored, sorted columns) from an edge list.

    The edge list must be free of self-loops and duplicates; ``ew`` gives the
    weight of each undirected edge and its dtype becomes the CSR value dtype.
    """
    eu = np.asarray(eu, dtype=np.int64)
    ev = np.asarray(ev, dtype=np.int64)
    ew = np.asarray(ew)
    order = np.lexsort((ev, eu))
    eu, ev, ew = eu[order], ev[order], ew[order]
    rows = np.concatenate([eu, ev])
    cols = np.concatenate([ev, eu])
    vals = np.concatenate([ew, ew])
    key = rows * n + cols
    perm = np.argsort(key, kind="stable")
    rows, cols, vals = rows[perm], cols[perm], vals[perm]
    counts = np.bincount(rows, minlength=n).astype(np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSRGraph(n=int(n), rowptr=rowptr, colidx=cols.astype(np.int32),
                    w=np.ascontiguousarray(vals), eu=eu, ev=ev, ew=ew, name=name)


def _relabel_keep(n: int, eu, ev, keep_mask):
    newid = np.full(n, -1, dtype=np.int64)
    newid[keep_mask] = np.arange(int(keep_mask.sum()), dtype=np.int64)
    sel = keep_mask[eu] & keep_mask[ev]
    return int(keep_mask.sum()), newid[eu[sel]], newid[ev[sel]], sel


def largest_component(n: int, eu: np.ndarray, ev: np.ndarray):
    """Restrict an edge list to its largest connected component.

    Nodes keep their relative order and are renumbered 0..n'-1.  Returns
    ``(n', eu', ev', edge_mask)``.
    """
    a = sp.coo_matrix((np.ones(eu.shape[0], dtype=np.int8), (eu, ev)), shape=(n, n)).tocsr()
    ncomp, lab = csg.connected_components(a, directed=True, connection="weak")
    if ncomp == 1:
        return n, eu, ev, np.ones(eu.shape[0], dtype=bool)
    sizes = np.bincount(lab)
    big = int(np.argmax(sizes))
    return _relabel_keep(n, eu, ev, lab == big)


# --------------------------------------------------------------------------- models

def erdos_renyi_gnm(n: int, m: int, rng: np.random.Generator):
    """G(n, m): m distinct undirected edges with uniform endpoints.

    Pairs are drawn in bulk; self-loops and repeats are discarded and more pairs
    drawn until m distinct edges exist (first-drawn edges are kept).
    """
    if m > n * (n - 1) // 2:
        raise ValueError("too many edges")
    eu = np.empty(0, dtype=np.int64)
    ev = np.empty(0, dtype=np.int64)
    need = m
    while need > 0:
        draw = int(need * 1.1) + 16
        u = rng.integers(0, n, size=draw)
        v = rng.integers(0, n, size=draw)
        eu, ev = _canonical_unique(np.concatenate([eu, u]), np.concatenate([ev, v]), n)
        need = m - eu.shape[0]
    return eu[:m], ev[:m]


def barabasi_albert(n: int, m: int, rng: np.random.Generator):
    """Barabasi-Albert preferential attachment.

    Seed graph: a star on nodes 0..m (centre 0).  Each new node t = m+1..n-1
    picks m distinct targets; each pick is uniform over a list that holds every
    node once per unit of its current degree (so picks are proportional to
    degree), repeats being redrawn.
    """
    if m < 1 or n <= m + 1:
        raise ValueError("need n > m + 1 >= 2")
    n_edges = m + m * (n - m - 1)
    eu = np.empty(n_edges, dtype=np.int64)
    ev = np.empty(n_edges, dtype=np.int64)
    eu[:m] = 0
    ev[:m] = np.arange(1, m + 1)
    rep = np.empty(2 * n_edges, dtype=np.int64)
    rep[:m] = 0
    rep[m:2 * m] = np.arange(1, m + 1)
    L = 2 * m
    e = m
    batch = 1 << 16
    pool = rng.random(batch)
    pi = 0
    rep_l = rep  # local alias
    for t in range(m + 1, n):
        chosen = []
        while len(chosen) < m:
            if pi == batch:
                pool = rng.random(batch)
                pi = 0
            c = int(rep_l[int(pool[pi] * L)])
            pi += 1
            if c not in chosen:
                chosen.append(c)
        eu[e:e + m] = t
        ev[e:e + m] = chosen
        e += m
        rep_l[L:L + m] = chosen
        rep_l[L + m:L + 2 * m] = t
        L += 2 * m
    return _canonical_unique(eu, ev, n)


def watts_strogatz(n: int, k: int, p: float, rng: np.random.Generator):
    """Watts-Strogatz small world.

    Ring lattice: node i is joined to i+1..i+k/2 (mod n).  Each lattice edge is
    selected for rewiring with probability p; a selected edge keeps its near end
    i and gets a uniform far end.  Rewired ends that make a self-loop or
    duplicate an existing edge are redrawn until the edge set is simple.
    """
    if k % 2 or k >= n:
        raise ValueError("k must be even and < n")
    h = k // 2
    base = np.repeat(np.arange(n, dtype=np.int64), h)
    off = np.tile(np.arange(1, h + 1, dtype=np.int64), n)
    u = base
    v = (base + off) % n
    sel = rng.random(u.shape[0]) < p
    v = v.copy()
    idx = np.nonzero(sel)[0]
    v[idx] = rng.integers(0, n, size=idx.shape[0])
    for _ in range(1000):
        a = np.minimum(u, v)
        b = np.maximum(u, v)
        key = a * n + b
        bad = a == b
        # duplicates: among identical keys keep an unrewired edge if any, else the first
        order = np.lexsort((sel.astype(np.int8), key))  # unrewired (False) first per key
        ks = key[order]
        dup_sorted = np.zeros(ks.shape[0], dtype=bool)
        dup_sorted[1:] = ks[1:] == ks[:-1]
        dup = np.zeros_like(dup_sorted)
        dup[order] = dup_sorted
        redo = (bad | dup) & sel
        if not redo.any():
            if (bad | dup).any():
                raise RuntimeError("lattice edge collided")
            break
        ridx = np.nonzero(redo)[0]
        v[ridx] = rng.integers(0, n, size=ridx.shape[0])
    else:
        raise RuntimeError("rewiring did not settle")
    return _canonical_unique(u, v, n)


def configuration_model_powerlaw(n: int, gamma: float, dmin: int, dmax: int,
                                 rng: np.random.Generator):
    """Erased configuration model with P(d) proportional to d^-gamma on [dmin, dmax].

    Degrees are drawn from the discrete power law by inverse CDF; if the degree
    sum is odd one node with degree < dmax gets one more stub.  Stubs are
    shuffled and paired consecutively, then self-loops and repeated edges are
    dropped ("erased").
    """
    d = np.arange(dmin, dmax + 1, dtype=np.float64)
    pmf = d ** (-gamma)
    cdf = np.cumsum(pmf)
    cdf /= cdf[-1]
    deg = (np.searchsorted(cdf, rng.random(n), side="right") + dmin).astype(np.int64)
    np.minimum(deg, dmax, out=deg)
    if deg.sum() % 2:
        cand = np.nonzero(deg < dmax)[0]
        deg[cand[int(rng.integers(0, cand.shape[0]))]] += 1
    stubs = np.repeat(np.arange(n, dtype=np.int64), deg)
    rng.shuffle(stubs)
    u = stubs[0::2]
    v = stubs[1::2]
    del stubs
    return _canonical_unique(u, v, n)


def stochastic_block_model(sizes, p_in: float, p_out: float, rng: np.random.Generator):
    """Stochastic block model with uniform in/out probabilities.

    For every block pair the number of edges is drawn from the binomial law of
    its possible pairs and that many distinct pairs are chosen uniformly.
    """
    sizes = [int(s) for s in sizes]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(offs[-1])
    us, vs = [], []
    for a in range(len(sizes)):
        for b in range(a, len(sizes)):
            if a == b:
                npairs = sizes[a] * (sizes[a] - 1) // 2
                p = p_in
            else:
                npairs = sizes[a] * sizes[b]
                p = p_out
            cnt = int(rng.binomial(npairs, p)) if npairs > 0 else 0
            if cnt == 0:
                continue
            if a == b:
                # cnt distinct unordered pairs inside the block, by rejection
                s = sizes[a]
                i_, j_ = erdos_renyi_gnm(s, cnt, rng)
                us.append(offs[a] + i_)
                vs.append(offs[a] + j_)
            else:
                picks = rng.choice(npairs, size=cnt, replace=False)
                us.append(offs[a] + picks // sizes[b])
                vs.append(offs[b] + picks % sizes[b])
    if not us:
        return n, np.empty(0, np.int64), np.empty(0, np.int64)
    eu, ev = _canonical_unique(np.concatenate(us), np.concatenate(vs), n)
    return n, eu, ev


# --------------------------------------------------------------------------- small graphs

def path_graph(n: int):
    return np.arange(n - 1, dtype=np.int64), np.arange(1, n, dtype=np.int64)


def cycle_graph(n: int):
    u = np.arange(n, dtype=np.int64)
    return _canonical_unique(u, (u + 1) % n, n)


def complete_graph(n: int):
    iu, iv = np.triu_indices(n, 1)
    return iu.astype(np.int64), iv.astype(np.int64)


def star_graph(n_leaves: int):
    return np.zeros(n_leaves, dtype=np.int64), np.arange(1, n_leaves + 1, dtype=np.int64)


def random_tree(n: int, rng: np.random.Generator):
    """Random recursive tree: node t attaches to a uniform earlier node."""
    parents = np.array([int(rng.integers(0, t)) for t in range(1, n)], dtype=np.int64)
    return parents, np.arange(1, n, dtype=np.int64)


def random_gnp_small(n: int, p: float, rng: np.random.Generator):
    iu, iv = np.triu_indices(n, 1)
    keep = rng.random(iu.shape[0]) < p
    return iu[keep].astype(np.int64), iv[keep].astype(np.int64)


def disjoint_union(graphs):
    """Concatenate graphs into one block-diagonal graph (node ids offset in order).

    Returns ``(union_graph, node_offsets)``; graph g occupies nodes
    ``node_offsets[g]:node_offsets[g+1]``.
    """
    offs = np.zeros(len(graphs) + 1, dtype=np.int64)
    for i, g in enumerate(graphs):
        offs[i + 1] = offs[i] + g.n
    eu = np.concatenate([g.eu + offs[i] for i, g in enumerate(graphs)])
    ev = np.concatenate([g.ev + offs[i] for i, g in enumerate(graphs)])
    ew = np.concatenate([g.ew for g in graphs])
    return csr_from_edges(int(offs[-1]), eu, ev, ew, name="union"), offs
