"""Seeded synthetic inputs shared by the tests, the benchmark and the
CPU-baseline runs.  This module holds no arithmetic of the method: it only
draws parameters and seeds.

Served mix (one request = one independent lattice): arrivals form a Poisson
process with exponential gaps of mean `gap_ms`; 70% are 2D Ising spin-1/2
with L log-uniform in [32, 2048] and T uniform in [1.5, 3.5], 30% are 2D
North-East with L log-uniform in [64, 4096] and c uniform in [0.05, 0.3];
sweeps are log-uniform in [10^3, 10^5]; every lattice starts random
(Ising) or at equilibrium (North-East).  numpy default_rng(99), one fixed
draw order per request: gap, model, L, T or c, sweeps, seed.  L is rounded
to the nearest even integer (the checkerboard needs even L).
"""
from __future__ import annotations

import math

import numpy as np


def served_mix(n=4096, seed=99, gap_ms=2.0, sweep_scale=1.0, round_to=2):
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        gap = rng.exponential(gap_ms) * 1e-3
        is_ne = rng.random() < 0.3
        lo, hi = (64, 4096) if is_ne else (32, 2048)
        L = math.exp(rng.uniform(math.log(lo), math.log(hi)))
        L = max(round_to, int(round(L / round_to)) * round_to)
        tc = rng.uniform(0.05, 0.3) if is_ne else rng.uniform(1.5, 3.5)
        sweeps = int(round(math.exp(rng.uniform(math.log(1e3), math.log(1e5)))))
        s = int(rng.integers(0, 2**63 - 1))
        t += gap
        out.append(dict(arrival=t, dims=2, L=L, two_S=1, model=1 if is_ne else 0,
                        J=0.0 if is_ne else 1.0, h=0.0, T_or_c=tc, seed=s,
                        init=2 if is_ne else 1,
                        sweeps=max(1, int(round(sweeps * sweep_scale)))))
    return out


def offered_updates(reqs):
    return sum(r["L"] ** 2 * r["sweeps"] for r in reqs)
