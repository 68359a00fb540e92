"""Seeded synthetic inputs shared by the library's callers, the tests and the
oracle side: measurement schedules and job lists.

This module holds no arithmetic of the growth method itself.  It only decides
WHEN widths are measured and WHICH jobs (L, N, t_max, seed) are run; both the
CUDA path and the CPU oracle consume these lists unchanged.
"""
from __future__ import annotations

import math

import numpy as np


def paper_schedule(t_max: int, m: float = 0.01, offset: float = 10.0, include_zero: bool = True):
    """Measurement times of Eq. 10: t_{i+1} = (t_i + offset) * exp(m), t_0 = 0.

    The paper's times are real numbers; widths are measured after whole sweeps,
    so each t_i is rounded up to an integer number of completed sweeps and
    repeated integers are dropped.  Times above ``t_max`` are not produced.
    """
    out = [0] if include_zero else []
    t = 0.0
    while True:
        t = (t + offset) * math.exp(m)
        T = int(math.ceil(t - 1e-9))
        if T > t_max:
            break
        if not out or T > out[-1]:
            out.append(T)
    return out


def log_schedule(t_max: int, n: int):
    """n log-spaced integer times from 1 to t_max: t_k = max(t_{k-1}+1,
    round(t_max ** (k / (n-1)))), k = 0..n-1 (used for the 40-point runs)."""
    out = []
    for k in range(n):
        T = int(round(t_max ** (k / (n - 1)))) if n > 1 else t_max
        if out and T <= out[-1]:
            T = out[-1] + 1
        out.append(T)
    if out[-1] > t_max:
        raise ValueError("n too large for t_max")
    return out


def pow2_schedule(t_max: int, include_zero: bool = True):
    """t = 0 (optional) and t = 2^k <= t_max."""
    out = [0] if include_zero else []
    k = 0
    while (1 << k) <= t_max:
        out.append(1 << k)
        k += 1
    return out


def batched_jobs(n_jobs: int = 256, seed: int = 2016, surfaces: int = 64):
    """Heterogeneous batch: L uniform in {256,...,4096}, N uniform in {1,2},
    t_max log-uniform integer in [1e3, 1e4], job seed = job index."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Ls = rng.choice([256, 512, 1024, 2048, 4096], size=n_jobs)
    Ns = rng.integers(1, 3, size=n_jobs)
    tm = np.rint(10 ** rng.uniform(3.0, 4.0, size=n_jobs)).astype(np.int64)
    return [dict(L=int(Ls[i]), N=int(Ns[i]), t_max=int(tm[i]), seed=i, surfaces=surfaces)
            for i in range(n_jobs)]


def served_jobs(n_jobs: int = 2000, rate: float = 50.0, seed: int = 2017, surfaces: int = 64):
    """Poisson request stream: arrival times (s) with mean rate ``rate``,
    L = 2^e with e uniform in 8..13, N uniform in 1..4, t_max log-uniform
    integer in [1e2, 1e4], job seed = request index."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=n_jobs)
    arrivals = np.cumsum(gaps)
    es = rng.integers(8, 14, size=n_jobs)
    Ns = rng.integers(1, 5, size=n_jobs)
    tm = np.rint(10 ** rng.uniform(2.0, 4.0, size=n_jobs)).astype(np.int64)
    return [dict(arrival=float(arrivals[i]), L=int(1 << int(es[i])), N=int(Ns[i]),
                 t_max=int(tm[i]), seed=i, surfaces=surfaces) for i in range(n_jobs)]
