"""Seeded node-vector pairs (x, y), one value per node.

Pair j of a workload is drawn from its own stream ``default_rng([seed, j])`` so any
subset of pairs can be regenerated without generating the others.  Outputs are
float64 arrays of shape [k, n] (one pair per row), the layout the library takes.
"""
from __future__ import annotations

import numpy as np


def _key(seed, j):
    """Seed sequence entropy for pair j: ``[*seed, j]`` (seed may be an int or a tuple)."""
    if isinstance(seed, (tuple, list)):
        return [int(s) for s in seed] + [int(j)]
    return [int(seed), int(j)]


def _sparse_uniform(n: int, frac: float, rng: np.random.Generator) -> np.ndarray:
    """Uniform[0,1) values on a random ``frac`` share of the nodes, zero elsewhere,
    normalised to sum 1 (support of at least one node)."""
    s = max(1, int(round(frac * n)))
    x = np.zeros(n, dtype=np.float64)
    idx = rng.choice(n, size=s, replace=False)
    vals = rng.random(s)
    while vals.sum() == 0.0:
        vals = rng.random(s)
    x[idx] = vals / vals.sum()
    return x


def sparse_uniform_pairs(n: int, k: int, frac: float, seed: int, first: int = 0):
    """Pairs of the "sparse uniform support" kind: x and y independently have
    Uniform[0,1) entries on a random ``frac`` of the nodes and sum to 1."""
    X = np.empty((k, n), dtype=np.float64)
    Y = np.empty((k, n), dtype=np.float64)
    for j in range(k):
        rng = np.random.default_rng(_key(seed, first + j))
        X[j] = _sparse_uniform(n, frac, rng)
        Y[j] = _sparse_uniform(n, frac, rng)
    return X, Y


def diffuse_uniform_pairs(n: int, k: int, seed: int, first: int = 0):
    """Diffuse pairs: x and y are Uniform[0,1) on every node, normalised to sum 1."""
    X = np.empty((k, n), dtype=np.float64)
    Y = np.empty((k, n), dtype=np.float64)
    for j in range(k):
        rng = np.random.default_rng(_key(seed, first + j))
        x = rng.random(n)
        y = rng.random(n)
        X[j] = x / x.sum()
        Y[j] = y / y.sum()
    return X, Y


def indicator_pairs(n: int, k: int, seed: int, first: int = 0):
    """Pairs x = e_i, y = e_j with i != j uniform (delta = e_i - e_j gives the
    effective resistance between i and j)."""
    X = np.zeros((k, n), dtype=np.float64)
    Y = np.zeros((k, n), dtype=np.float64)
    ij = np.empty((k, 2), dtype=np.int64)
    for j in range(k):
        rng = np.random.default_rng(_key(seed, first + j))
        a = int(rng.integers(0, n))
        b = int(rng.integers(0, n - 1))
        if b >= a:
            b += 1
        X[j, a] = 1.0
        Y[j, b] = 1.0
        ij[j] = (a, b)
    return X, Y, ij
