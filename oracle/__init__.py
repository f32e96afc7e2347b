"""Oracle for the Generalized Euclidean (GE) node-vector distance -- TEST INFRASTRUCTURE.

This package is the slow, plain, obviously-correct CPU statement of what the
library computes.  It exists only to check the CUDA path: nothing in the product
(the ``paper_2310_11222_gb300`` package, its C ABI or its kernels) may import,
link or call it.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the CUDA path; the two meet
only in the seeded input generators of ``synth/``.

What it computes (Section 3.1 of the paper, the GE equation):

    d(a, b)^2 = (a - b)^T  L^+  (a - b),   L = D - W,  L^+ the Moore-Penrose pseudoinverse,

for an undirected graph with positive weights.  Two routes:

* ``oracle.dense`` -- forms L^+ by a dense FP64 symmetric eigendecomposition (the
  costly route the paper replaces, Section 3.1), plus an independent second dense
  route through the grounded Laplacian and a Cholesky factorisation; also the
  dense gradient of d^2 with respect to the vectors and the edge weights, the
  effective resistance of node-id pairs (the GE equation on indicator vectors)
  and the network variance (1/2) sum_ij p_i p_j R(i, j) of node weights.
* ``oracle.cg`` -- a plain C FP64 Jacobi-preconditioned conjugate gradient on the
  sparse Laplacian (the "CG" Laplacian solver of Section 3.2 and Table 1), for
  graphs too large for the dense route.

Readings of points the paper leaves open (each is also listed in the design notes):

* weights: L_uv = -w_uv, L_uu = sum_v w_uv, built from W_sym = (W + W^T)/2 of the
  stored entries; self-loops are dropped, repeated entries summed;
* disconnected graphs: L^+ annihilates per-component constants, so the result
  is (P delta)^T L^+ (P delta) with P the per-component mean-zero projector;
  exactly c zero eigenvalues are dropped, c = number of connected components;
* d = sqrt(max(d^2, 0));
* effective resistance between different components: +inf (no current flows).
"""
