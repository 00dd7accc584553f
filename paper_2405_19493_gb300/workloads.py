"""Seeded synthetic inputs shared by the tests, the bench and the oracle calls.

Holds none of the method's arithmetic: only seeds, stream lengths and request
parameters, with the shapes of the workloads the library is measured on.

  * correctness workload: 64 streams x 16,384 variates, seeds 0x5EED + s;
  * bulk workload: 2^20 streams x 1,024 variates (2^30 outputs), seeds 0x5EED + s;
  * batched workload: 10,000 streams, lengths log-uniform in [1, 2^20]
    (L = clip(round(2^(20 u)), 1, 2^20), u from numpy default_rng(7));
  * mutation requests: populations P x L (P log-uniform 16..4096, L log-uniform
    8..100,000), sigma uniform in [0.01, 1], per-request seed, Poisson arrivals.
"""

from __future__ import annotations

import numpy as np

SEED_BASE = 0x5EED


def seeds(n: int, base: int = SEED_BASE) -> np.ndarray:
    return (np.uint64(base) + np.arange(n, dtype=np.uint64)).astype(np.uint64)


def batched_lengths(n: int = 10_000, seed: int = 7, max_log2: int = 20) -> np.ndarray:
    u = np.random.default_rng(seed).random(n)
    L = np.rint(np.exp2(max_log2 * u))
    return np.clip(L, 1, 2 ** max_log2).astype(np.uint64)


def log_uniform_int(rng, lo: int, hi: int, size=None):
    return np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size))).astype(np.int64)


def mutation_requests(n: int, rate_hz: float, seed: int = 11, p_range=(16, 4096),
                      l_range=(8, 100_000), max_elems: int | None = None,
                      generate_frac: float = 0.0):
    """n requests: dicts with P, L, sigma, seed, arrival (seconds) and kind
    ("mutate", or "generate" for about generate_frac of them)."""
    rng = np.random.default_rng(seed)
    P = log_uniform_int(rng, *p_range, size=n)
    L = log_uniform_int(rng, *l_range, size=n)
    if max_elems is not None:
        over = P * L > max_elems
        L = np.where(over, np.maximum(1, max_elems // P), L)
    sigma = rng.uniform(0.01, 1.0, size=n)
    rseed = rng.integers(0, 2 ** 63, size=n, dtype=np.int64)
    arrival = np.cumsum(rng.exponential(1.0 / rate_hz, size=n))
    gen = rng.random(n) < generate_frac if generate_frac > 0 else np.zeros(n, dtype=bool)
    return [dict(P=int(P[k]), L=int(L[k]), sigma=float(sigma[k]), seed=int(rseed[k]),
                 arrival=float(arrival[k]), kind="generate" if gen[k] else "mutate")
            for k in range(n)]
