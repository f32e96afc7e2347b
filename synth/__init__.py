"""Seeded synthetic inputs shared by the oracle-side tests, the GPU tests and the bench.

This package only *generates* inputs: random graphs (as symmetric CSR adjacency),
edge weights and node-vector pairs.  It contains none of the method's arithmetic
(no Laplacian, no degree, no projection, no solve), so the oracle and the CUDA
path can both consume its output without sharing any computation.

The graph models follow the outlines of Section 4.1.2 of the paper (Erdos-Renyi
G(n,m), Barabasi-Albert, Watts-Strogatz, stochastic block model) plus the erased
configuration model with a power-law degree sequence used by the heavy-tailed
workload.  Where the paper only gives an outline, the concrete rule is stated in
each generator's docstring.
"""
from .graphs import (CSRGraph, erdos_renyi_gnm, barabasi_albert, watts_strogatz,
                     configuration_model_powerlaw, stochastic_block_model,
                     largest_component, csr_from_edges, disjoint_union,
                     path_graph, cycle_graph, complete_graph, star_graph,
                     random_tree, random_gnp_small)
from .vectors import sparse_uniform_pairs, diffuse_uniform_pairs, indicator_pairs
from .workloads import (workload_ba_small, workload_er_large, workload_batched,
                        workload_powerlaw, workload_grad, sweep_graph, WORKLOADS)

__all__ = [
    "CSRGraph", "erdos_renyi_gnm", "barabasi_albert", "watts_strogatz",
    "configuration_model_powerlaw", "stochastic_block_model", "largest_component",
    "csr_from_edges", "disjoint_union", "path_graph", "cycle_graph", "complete_graph",
    "star_graph", "random_tree", "random_gnp_small", "sparse_uniform_pairs",
    "diffuse_uniform_pairs", "indicator_pairs", "workload_ba_small", "workload_er_large",
    "workload_batched", "workload_powerlaw", "workload_grad", "sweep_graph", "WORKLOADS",
]
