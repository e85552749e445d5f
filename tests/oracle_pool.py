"""Oracle runs in worker processes, for the full-size parity tests.

The oracle is single-threaded; a few long runs (10^8 - 10^9 site updates
each) are spread over a spawn-started process pool so that they overlap
with each other and with the GPU work of the test.  Spawn (not fork), so
the workers never inherit a CUDA context.
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os


def run_oracle(dims, L, two_S, model, J, h, T_or_c, seed, init, n):
    """n oracle sweeps from the initial state: (spins, flags, series)."""
    import oracle
    o = oracle.Lattice(dims, L, two_S, model, J, h, T_or_c, seed=seed, init=init)
    ser = o.sweep(n)
    return o.spins, o.flags, ser


def pool(workers: int):
    n = max(1, min(workers, os.cpu_count() or 1))
    return cf.ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn"))
