"""Seeded synthetic inputs shared by the tests and the benchmark.

This module draws random numbers only; it contains none of the method's
arithmetic.  Both the CUDA path and the CPU oracle receive the same arrays.
Generators: numpy ``PCG64(seed)``.
"""
from __future__ import annotations

import math

import numpy as np

INF16 = 0x7FFF
INF8 = 0xFF


def block_inf_matrix(rows: int, cols: int, seed: int, dtype=np.int16, inf_frac: float = 0.4,
                     block: int = 128, lo: int = 0, hi: int = 31) -> np.ndarray:
    """Entries i.i.d. uniform in [lo, hi]; each block x block tile (partial at
    the edges) is set entirely to INF with probability inf_frac."""
    rng = np.random.Generator(np.random.PCG64(seed))
    inf = INF16 if np.dtype(dtype) == np.int16 else INF8
    X = rng.integers(lo, hi + 1, size=(rows, cols), dtype=dtype)
    br, bc = math.ceil(rows / block), math.ceil(cols / block)
    mask = rng.random((br, bc)) < inf_frac
    for i, j in zip(*np.nonzero(mask)):
        X[i * block:(i + 1) * block, j * block:(j + 1) * block] = inf
    return X


def entry_inf_matrix(rows: int, cols: int, seed: int, dtype=np.int16, inf_frac: float = 0.3,
                     lo: int = 0, hi: int = 31) -> np.ndarray:
    """Entries uniform in [lo, hi], each INF independently with prob inf_frac."""
    rng = np.random.Generator(np.random.PCG64(seed))
    inf = INF16 if np.dtype(dtype) == np.int16 else INF8
    X = rng.integers(lo, hi + 1, size=(rows, cols), dtype=dtype)
    X[rng.random((rows, cols)) < inf_frac] = inf
    return X


def batch_sizes(count: int = 96, lo: int = 64, hi: int = 8192, seed: int = 7) -> list:
    """Square sizes N = round(exp(U[ln lo, ln hi])), one per product."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.uniform(math.log(lo), math.log(hi), size=count)
    return [int(round(math.exp(x))) for x in u]


def serving_queries(count: int = 10000, seed: int = 11, n_lo: int = 2, n_hi: int = 10,
                    m_lo: int = 3, m_hi: int = 2000):
    """(n, m) queries: n uniform in {n_lo..n_hi}, m = round(exp(U[ln m_lo, ln m_hi]))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = rng.integers(n_lo, n_hi + 1, size=count)
    m = np.rint(np.exp(rng.uniform(math.log(m_lo), math.log(m_hi), size=count))).astype(np.int64)
    return n.astype(np.int64), m


def poisson_arrivals(count: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process with the given rate."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))
