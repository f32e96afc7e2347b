"""The five seeded workloads (graph + vector pairs) with the paper's workload shapes.

Seeds: graph seed 1000 + i and vector seed 2000 + i for workload i.  Every
builder takes ``scale`` (multiplies the node count) so tests can run the same
recipe at a size a CPU finishes in seconds.  The recipes:

0. ``ba_small``   Barabasi-Albert n=2,000, m=3, unit weights; 16 pairs with Uniform
   support on 10% of nodes, normalised.  FP64 PCG to relative residual 1e-10.
1. ``er_large``   Erdos-Renyi n=1,000,000, m=5,000,000 (mean degree 10), largest
   component, weights Uniform[0.5, 2) FP64; 8 pairs with 1% support, solved
   one right-hand side at a time in FP64.
2. ``batched``    64 graphs with node counts log-uniform in [1e3, 2e5]; graphs 0..31
   Barabasi-Albert with m uniform in {2..6}, graphs 32..63 Watts-Strogatz k=10,
   p=0.1 (largest component), unit FP32 weights; per graph 16 pairs e_i - e_j and
   16 diffuse normalised Uniform pairs.
3. ``powerlaw``   erased configuration model, n=10,000,000, P(d) ~ d^-2.3 on
   [2, 10,000], largest component, lognormal(0,1) FP32 weights; 128 pairs with
   0.1% support.
4. ``grad``       Barabasi-Albert n=1,000,000, m=5, lognormal(0,0.5) FP32 weights;
   64 pairs with 10% support; d^2 and its gradients.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

from .graphs import (CSRGraph, barabasi_albert, configuration_model_powerlaw,
                     csr_from_edges, disjoint_union, erdos_renyi_gnm, largest_component,
                     stochastic_block_model, watts_strogatz)
from .vectors import diffuse_uniform_pairs, indicator_pairs, sparse_uniform_pairs


@dataclass
class Workload:
    name: str
    index: int
    graph: CSRGraph
    k: int
    pairs: Callable[[int, int], tuple] = field(repr=False)
    """pairs(first, count) -> (X, Y) float64 [count, n] for pairs first..first+count-1"""
    wdtype: type = np.float64
    graphs: Optional[List[CSRGraph]] = field(default=None, repr=False)
    node_offsets: Optional[np.ndarray] = field(default=None, repr=False)
    meta: dict = field(default_factory=dict)


def _weights(kind: str, m: int, rng: np.random.Generator, dtype):
    if kind == "unit":
        return np.ones(m, dtype=dtype)
    if kind == "uniform_0.5_2":
        return rng.uniform(0.5, 2.0, size=m).astype(dtype)
    if kind.startswith("lognormal_"):
        sigma = float(kind.split("_")[1])
        return rng.lognormal(0.0, sigma, size=m).astype(dtype)
    raise ValueError(kind)


def workload_ba_small(scale: float = 1.0) -> Workload:
    i = 0
    n = max(16, int(round(2000 * scale)))
    rng = np.random.default_rng(1000 + i)
    eu, ev = barabasi_albert(n, 3, rng)
    g = csr_from_edges(n, eu, ev, _weights("unit", eu.shape[0], rng, np.float64), name="ba_small")
    return Workload("ba_small", i, g, 16,
                    lambda f, c: sparse_uniform_pairs(n, c, 0.10, 2000 + i, f), np.float64,
                    meta={"rtol": 1e-10, "mode": "fp64"})


def workload_er_large(scale: float = 1.0) -> Workload:
    i = 1
    n0 = max(64, int(round(1_000_000 * scale)))
    rng = np.random.default_rng(1000 + i)
    eu, ev = erdos_renyi_gnm(n0, 5 * n0, rng)
    n, eu, ev, _ = largest_component(n0, eu, ev)
    g = csr_from_edges(n, eu, ev, _weights("uniform_0.5_2", eu.shape[0], rng, np.float64),
                       name="er_large")
    return Workload("er_large", i, g, 8,
                    lambda f, c: sparse_uniform_pairs(n, c, 0.01, 2000 + i, f), np.float64,
                    meta={"rtol": 1e-10, "mode": "fp64", "single_rhs": True, "n_generated": n0})


def batched_graph(gidx: int, scale: float = 1.0) -> CSRGraph:
    """Graph ``gidx`` (0..63) of the batched workload."""
    i = 2
    sizes_rng = np.random.default_rng(1000 + i)
    logn = sizes_rng.uniform(np.log(1e3), np.log(2e5), size=64)
    ms = sizes_rng.integers(2, 7, size=64)
    n = max(32, int(round(np.exp(logn[gidx]) * scale)))
    rng = np.random.default_rng([1000 + i, gidx])
    if gidx < 32:
        eu, ev = barabasi_albert(n, int(ms[gidx]), rng)
        kind = f"ba_m{int(ms[gidx])}"
    else:
        eu, ev = watts_strogatz(n, 10, 0.1, rng)
        n, eu, ev, _ = largest_component(n, eu, ev)
        kind = "ws_k10_p0.1"
    g = csr_from_edges(n, eu, ev, np.ones(eu.shape[0], dtype=np.float32), name=kind)
    return g


def batched_pairs(g: CSRGraph, gidx: int):
    """The 32 pairs of graph ``gidx``: 16 indicator pairs then 16 diffuse pairs."""
    i = 2
    Xa, Ya, _ = indicator_pairs(g.n, 16, (2000 + i, gidx, 0))
    Xb, Yb = diffuse_uniform_pairs(g.n, 16, (2000 + i, gidx, 1))
    return np.concatenate([Xa, Xb]), np.concatenate([Ya, Yb])


def workload_batched(scale: float = 1.0, n_graphs: int = 64) -> Workload:
    graphs = [batched_graph(gi, scale) for gi in range(n_graphs)]
    union, offs = disjoint_union(graphs)

    def pairs(first, count):
        assert first == 0 and count == 32
        Xs, Ys = [], []
        for gi, g in enumerate(graphs):
            X, Y = batched_pairs(g, gi)
            Xs.append(X)
            Ys.append(Y)
        return Xs, Ys

    return Workload("batched", 2, union, 32, pairs, np.float32, graphs=graphs,
                    node_offsets=offs, meta={"rtol": 1e-6, "mode": "fp32"})


def workload_powerlaw(scale: float = 1.0) -> Workload:
    i = 3
    n0 = max(64, int(round(10_000_000 * scale)))
    dmax = max(4, min(10_000, n0 // 10))
    rng = np.random.default_rng(1000 + i)
    eu, ev = configuration_model_powerlaw(n0, 2.3, 2, dmax, rng)
    n, eu, ev, _ = largest_component(n0, eu, ev)
    g = csr_from_edges(n, eu, ev, _weights("lognormal_1.0", eu.shape[0], rng, np.float32),
                       name="powerlaw")
    return Workload("powerlaw", i, g, 128,
                    lambda f, c: sparse_uniform_pairs(n, c, 0.001, 2000 + i, f), np.float32,
                    meta={"rtol_d2": 1e-8, "mode": "mixed", "n_generated": n0, "dmax": dmax})


def workload_grad(scale: float = 1.0) -> Workload:
    i = 4
    n = max(64, int(round(1_000_000 * scale)))
    rng = np.random.default_rng(1000 + i)
    eu, ev = barabasi_albert(n, 5, rng)
    g = csr_from_edges(n, eu, ev, _weights("lognormal_0.5", eu.shape[0], rng, np.float32),
                       name="grad")
    return Workload("grad", i, g, 64,
                    lambda f, c: sparse_uniform_pairs(n, c, 0.10, 2000 + i, f), np.float32,
                    meta={"mode": "fp32"})


WORKLOADS = {
    "ba_small": workload_ba_small,
    "er_large": workload_er_large,
    "batched": workload_batched,
    "powerlaw": workload_powerlaw,
    "grad": workload_grad,
}


def sweep_graph(model: str, n: int, mean_degree: float, seed: int) -> CSRGraph:
    """Unit-weight graph of the size and density sweeps (the paper's synthetic models,
    compared at the same number of edges n * mean_degree / 2):
      er   G(n, m) with m = n * mean_degree / 2;
      ba   Barabasi-Albert with mean_degree / 2 edges per new node (at least 1);
      ws   Watts-Strogatz ring with mean_degree neighbours (even, at least 2), p = 0.1;
      sbm  10 equal groups, 80% of a node's expected edges inside its group.
    The whole graph is kept (components included)."""
    rng = np.random.default_rng([4000, seed])
    if model == "er":
        m = max(1, int(round(n * mean_degree / 2)))
        eu, ev = erdos_renyi_gnm(n, m, rng)
    elif model == "ba":
        eu, ev = barabasi_albert(n, max(1, int(round(mean_degree / 2))), rng)
    elif model == "ws":
        k = max(2, 2 * int(round(mean_degree / 2)))
        eu, ev = watts_strogatz(n, k, 0.1, rng)
    elif model == "sbm":
        groups = 10
        size = n // groups
        sizes = [size] * (groups - 1) + [n - size * (groups - 1)]
        p_in = min(1.0, 0.8 * mean_degree / max(size - 1, 1))
        p_out = min(1.0, 0.2 * mean_degree / max(n - size, 1))
        _, eu, ev = stochastic_block_model(sizes, p_in, p_out, rng)
    else:
        raise ValueError(model)
    return csr_from_edges(n, eu, ev, np.ones(len(eu)), name=f"{model}_{n}_{mean_degree}")
