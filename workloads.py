"""Seeded synthetic workloads (query lists) for BBP digit extraction.

This module only draws positions, precisions and arrival times; it holds none of
the method's arithmetic, and both the oracle-side and the GPU-side tests and
benchmarks take their inputs from here.

* batched: n = floor(10^U(lo, hi)), P uniform in {64, 128, 256} (seed 0, 4096
  queries, lo = 4, hi = 10 for the full batched configuration).
* serving: Poisson arrivals (exponential gaps at a given rate), n = floor(10^U(6,
  11)), P uniform in {64, 256} (seed 1), plus optionally one long query
  (n = 1e13, P = 256) submitted at t = 0.
"""

from __future__ import annotations

import numpy as np


def batched_queries(count: int = 4096, seed: int = 0, lo: float = 4.0, hi: float = 10.0,
                    precisions=(64, 128, 256)) -> tuple[list[int], list[int]]:
    rng = np.random.default_rng(seed)
    ns = np.floor(10.0 ** rng.uniform(lo, hi, count)).astype(np.int64)
    Ps = rng.choice(np.asarray(precisions, dtype=np.int64), count)
    return [int(v) for v in ns], [int(v) for v in Ps]


def expected_terms(ns, step_fraction: float = 0.7) -> float:
    """About 0.7 n terms per query for Bellard's formula (7 series, n/10 each)."""
    return float(sum(step_fraction * n for n in ns))


def serving_arrivals(count: int, rate_per_s: float, seed: int = 1, lo: float = 6.0, hi: float = 11.0,
                     precisions=(64, 256), long_query: tuple[int, int] | None = None):
    """[(arrival_time_s, n, P)], sorted by time; the long query (if any) arrives at 0."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, count)
    times = np.cumsum(gaps)
    ns = np.floor(10.0 ** rng.uniform(lo, hi, count)).astype(np.int64)
    Ps = rng.choice(np.asarray(precisions, dtype=np.int64), count)
    out = [(float(t), int(n), int(P)) for t, n, P in zip(times, ns, Ps)]
    if long_query is not None:
        out.insert(0, (0.0, int(long_query[0]), int(long_query[1])))
    return out
