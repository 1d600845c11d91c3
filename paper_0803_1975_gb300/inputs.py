"""Seeded synthetic inputs for the GF(p) products.

This module only draws random residues; it holds none of the method's
arithmetic, so both the library's tests/benchmark and the CPU oracle can take
their inputs from it.  Every generator is numpy's PCG64 seeded with
1000 * workload + trial, so a workload is reproducible from two integers.

Workloads (the paper has no dataset; these stand in for its experiments):

1. plain product, p = 3, m = k = n = 256, residues i.i.d. uniform in [0, p);
2. Q-adic compressed product, p = 3, m = k = n = 1024, uniform residues;
3. exact tensor-core product, p in {3, 31, 251}, m = k = n = 8192;
4. 4096 independent squares A_i^2 mod p_i of symmetric 0/1 adjacency
   matrices (zero diagonal, edge density 0.5), n_i log-uniform in [16, 512],
   p_i uniform in {3, 5, 7} -- the strongly regular graph computations that
   motivate the paper (Section 1);
5. all forms at p = 5, m = k = n = 16384, uniform residues.
"""
from __future__ import annotations

import math

import numpy as np


def rng(workload: int, trial: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(1000 * workload + trial))


def residues(g: np.random.Generator, p: int, rows: int, cols: int) -> np.ndarray:
    """rows x cols uint8 residues i.i.d. uniform in [0, p)."""
    return g.integers(0, p, size=(rows, cols), dtype=np.uint8)


def adjacency(g: np.random.Generator, n: int, density: float = 0.5) -> np.ndarray:
    """Symmetric 0/1 matrix with zero diagonal; each edge of the upper
    triangle is present with probability `density`."""
    upper = np.triu(g.random((n, n)) < density, k=1)
    return (upper | upper.T).astype(np.uint8)


def batched_sizes(g: np.random.Generator, count: int, nmin: int = 16, nmax: int = 512):
    """n_i = round(exp(U(ln nmin, ln nmax))), clipped to [nmin, nmax]."""
    x = np.exp(g.uniform(math.log(nmin), math.log(nmax), size=count))
    return np.clip(np.rint(x).astype(np.int64), nmin, nmax)


def batched_problems(workload: int = 4, trial: int = 0, count: int = 4096, nmin: int = 16,
                     nmax: int = 512, primes=(3, 5, 7)):
    """The batched workload: a list of (p_i, A_i) with A_i an n_i x n_i
    adjacency matrix; the product asked for is A_i @ A_i mod p_i."""
    g = rng(workload, trial)
    ns = batched_sizes(g, count, nmin, nmax)
    ps = g.choice(np.asarray(primes, dtype=np.int64), size=count)
    return [(int(p), adjacency(g, int(n))) for p, n in zip(ps, ns)]


def near_max(p: int, rows: int, cols: int) -> np.ndarray:
    """All entries p - 1: the largest possible dot products."""
    return np.full((rows, cols), p - 1, dtype=np.uint8)
