"""Dense FP64 routes to the GE distance (test infrastructure; see ``oracle/__init__``).

* ``laplacian_dense``      L = D - W from the stored CSR entries (Section 3.1).
* ``components``           connected components by breadth-first search.
* ``pinv_laplacian``       L^+ by symmetric eigendecomposition with exactly c zero
                           eigenvalues dropped (Section 3.1: "SVD" of L; for a
                           symmetric positive semidefinite L the SVD is its
                           eigendecomposition).
* ``ge_d2_eig``            d^2 = delta^T L^+ delta   (Section 3.1, GE equation).
* ``ge_d2_grounded``       the same number by an independent route: per component,
                           ground one node, Cholesky-solve the reduced system.
* ``ge_grad_dense``        gradients of d^2 from z = L^+ delta.
* ``effective_resistance`` R(u, v) on node-id pairs (indicator vectors), +inf
                           across components.
* ``network_variance``     (1/2) sum_ij p_i p_j R(i, j) of node weights p.

Parity is pinned by closed forms (effective resistances of paths, cycles, trees,
stars and complete graphs), Foster's theorem, invariants and the agreement of the
two independent dense routes; see ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

from collections import deque

import numpy as np
import scipy.linalg as sla


def laplacian_dense(n, rowptr, colidx, w):
    """Dense FP64 Laplacian from CSR adjacency entries.

    Each stored entry (u, v, w) with u != v contributes w/2 to the symmetric pair
    (u,v)/(v,u): the operator is built from W_sym = (W + W^T)/2, so a symmetric
    CSR (both directions stored) gives L_uv = -w_uv and L_uu = sum_v w_uv.
    Self-loops are ignored (they cancel in D - W); repeated entries add up.
    """
    L = np.zeros((n, n), dtype=np.float64)
    rowptr = np.asarray(rowptr, dtype=np.int64)
    for u in range(n):
        for e in range(int(rowptr[u]), int(rowptr[u + 1])):
            v = int(colidx[e])
            if v == u:
                continue
            h = 0.5 * float(w[e])
            L[u, v] -= h
            L[v, u] -= h
            L[u, u] += h
            L[v, v] += h
    return L


def components(n, rowptr, colidx):
    """Connected-component labels 0..c-1 (numbered by smallest node) via BFS.

    Edges are followed in both directions, so the result is correct even for a
    CSR that stores only one direction of some edges.
    """
    adj = [[] for _ in range(n)]
    for u in range(n):
        for e in range(int(rowptr[u]), int(rowptr[u + 1])):
            v = int(colidx[e])
            if v != u:
                adj[u].append(v)
                adj[v].append(u)
    lab = np.full(n, -1, dtype=np.int64)
    c = 0
    for s in range(n):
        if lab[s] >= 0:
            continue
        lab[s] = c
        q = deque([s])
        while q:
            x = q.popleft()
            for y in adj[x]:
                if lab[y] < 0:
                    lab[y] = c
                    q.append(y)
        c += 1
    return lab, c


def project_mean_zero(delta, lab, c):
    """Per-component mean-zero projection P delta (delta: [k, n] or [n])."""
    d = np.array(delta, dtype=np.float64, copy=True)
    one = d.ndim == 1
    if one:
        d = d[None, :]
    for comp in range(c):
        idx = np.nonzero(lab == comp)[0]
        d[:, idx] -= d[:, idx].mean(axis=1, keepdims=True)
    return d[0] if one else d


def pinv_laplacian(L, c):
    """Moore-Penrose pseudoinverse of a graph Laplacian by eigendecomposition.

    The c smallest eigenvalues (c = number of connected components, the dimension
    of the null space of L) are treated as exactly zero; every other eigenvalue
    is inverted.  L^+ = V diag(lambda^+) V^T.
    """
    lam, V = np.linalg.eigh(L)
    inv = np.zeros_like(lam)
    inv[c:] = 1.0 / lam[c:]
    return (V * inv) @ V.T


def ge_d2_eig(n, rowptr, colidx, w, X, Y):
    """d^2 = (x-y)^T L^+ (x-y) for each row pair of X, Y ([k, n]) -- GE equation, Section 3.1."""
    L = laplacian_dense(n, rowptr, colidx, w)
    _, c = components(n, rowptr, colidx)
    Lp = pinv_laplacian(L, c)
    D = np.atleast_2d(np.asarray(X, np.float64) - np.asarray(Y, np.float64))
    return np.einsum("ki,ij,kj->k", D, Lp, D)


def ge_d2_grounded(n, rowptr, colidx, w, X, Y):
    """Second dense route: grounded-Laplacian Cholesky.

    For each component ground its smallest node r (delete row and column r).
    The reduced matrix is symmetric positive definite; with delta projected
    mean-zero per component, z~ = L~^{-1} delta~ extended by z_r = 0 satisfies
    L z = P delta, so d^2 = delta~^T z~ equals (P delta)^T L^+ (P delta).
    """
    L = laplacian_dense(n, rowptr, colidx, w)
    lab, c = components(n, rowptr, colidx)
    D = project_mean_zero(np.atleast_2d(np.asarray(X, np.float64) - np.asarray(Y, np.float64)),
                          lab, c)
    grounded = np.zeros(n, dtype=bool)
    for comp in range(c):
        grounded[np.nonzero(lab == comp)[0][0]] = True
    keep = ~grounded
    if not keep.any():
        return np.zeros(D.shape[0])
    Lr = L[np.ix_(keep, keep)]
    cf = sla.cho_factor(Lr, lower=True)
    Dr = D[:, keep]
    Z = sla.cho_solve(cf, Dr.T).T
    return np.einsum("ki,ki->k", Dr, Z)


def effective_resistance(n, rowptr, colidx, w, U, V):
    """R(u, v) = (e_u - e_v)^T L^+ (e_u - e_v) for node-id pairs (the GE equation of
    Section 3.1 on indicator vectors), from the dense L^+ of each component.  With
    no path between u != v the resistance is infinite (no current flows); u = v
    gives 0."""
    L = laplacian_dense(n, rowptr, colidx, w)
    lab, c = components(n, rowptr, colidx)
    Lp = pinv_laplacian(L, c)
    out = np.empty(len(U))
    for t, (u, v) in enumerate(zip(np.asarray(U, np.int64), np.asarray(V, np.int64))):
        if u == v:
            out[t] = 0.0
        elif lab[u] != lab[v]:
            out[t] = np.inf
        else:
            out[t] = Lp[u, u] + Lp[v, v] - 2.0 * Lp[u, v]
    return out


def network_variance(n, rowptr, colidx, w, nodes, p):
    """Network variance of the node weights p on the nodes ``nodes`` (a distribution
    on the graph, as in the variance of distributions on graphs the paper cites in
    Section 2): (1/2) sum_ij p_i p_j R(i, j), R the effective resistance; +inf when
    mass sits on two components."""
    nodes = np.asarray(nodes, np.int64)
    p = np.asarray(p, np.float64)
    a, b = np.meshgrid(nodes, nodes, indexing="ij")
    R = effective_resistance(n, rowptr, colidx, w, a.ravel(), b.ravel()).reshape(len(nodes), -1)
    P = np.outer(p, p)
    mass = P > 0
    if np.isinf(R[mass]).any():
        return np.inf
    return 0.5 * float(np.sum(P[mass] * R[mass]))


def ge_z_dense(n, rowptr, colidx, w, X, Y):
    """z = L^+ (x - y) per pair ([k, n]); mean-zero per component by construction."""
    L = laplacian_dense(n, rowptr, colidx, w)
    _, c = components(n, rowptr, colidx)
    Lp = pinv_laplacian(L, c)
    D = np.atleast_2d(np.asarray(X, np.float64) - np.asarray(Y, np.float64))
    return D @ Lp  # L^+ symmetric


def ge_grad_dense(n, rowptr, colidx, w, X, Y, gbar):
    """Gradients of  sum_p gbar_p d_p^2  with z_p = L^+ delta_p.

    * d(d^2)/dx = 2 z,  d(d^2)/dy = -2 z   (L^+ symmetric);
    * per stored CSR entry (u, v):  -1/2 * sum_p gbar_p (z_pu - z_pv)^2, from
      dL^+ = -L^+ dL L^+ and dL/dW_uv = 1/2 (e_u - e_v)(e_u - e_v)^T under the
      W_sym reading (an undirected edge stored twice therefore collects
      -(z_u - z_v)^2 in total).
    Returns (grad_w [nnz], grad_x [k, n], grad_y [k, n]).
    """
    Z = ge_z_dense(n, rowptr, colidx, w, X, Y)
    gbar = np.asarray(gbar, dtype=np.float64).reshape(-1)
    rows = np.repeat(np.arange(n), np.diff(np.asarray(rowptr, dtype=np.int64)))
    cols = np.asarray(colidx, dtype=np.int64)
    diff = Z[:, rows] - Z[:, cols]
    gw = -0.5 * np.einsum("k,ke->e", gbar, diff * diff)
    gw[rows == cols] = 0.0
    gx = 2.0 * gbar[:, None] * Z
    return gw, gx, -gx
