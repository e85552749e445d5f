"""Full-size parity: the benchmarked lattices against the CPU oracle.

2D Ising spin-1/2 at L = 4096 (random start, seed 7) at each benchmarked
temperature T in {2.0, 2.269185, 3.0}, in both spin layouts (int8 through
the kernel the autotuner picks and through each fixed kernel, bit-packed),
for 100 sweeps in the launch configuration the benchmark uses (graph
replays); the North-East model at L = 8192 (c = 0.3, equilibrium start,
seed 21) and 3D spin-1 at L = 256 (seed 11) for 10 sweeps.  Spins,
persistence flags and every per-sweep counter must be identical: integer
work, zero tolerance.  The oracle runs (10^8 - 10^9 updates each) are made
in parallel worker processes while the GPU runs.
"""
import numpy as np
import pytest

import paper_1209_0296_gb300 as lt
from tests.oracle_pool import pool, run_oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TEMPS = (2.0, 2.269185, 3.0)
N_2D = 100
N_OTHER = 10
CASES = {("ising", T): (2, 4096, 1, lt.ISING, 1.0, 0.0, T, 7, lt.INIT_RANDOM, N_2D) for T in TEMPS}
CASES[("ne", 0.3)] = (2, 8192, 1, lt.NE, 0.0, 0.0, 0.3, 21, lt.INIT_EQUILIBRIUM, N_OTHER)
CASES[("3d", 2.0 + 7 * 2.0 / 15)] = (3, 256, 2, lt.ISING, 1.0, 0.0, 2.0 + 7 * 2.0 / 15, 11, lt.INIT_RANDOM, N_OTHER)


@pytest.fixture(scope="module")
def oracle_runs():
    ex = pool(len(CASES))
    futs = {key: ex.submit(run_oracle, *args) for key, args in CASES.items()}
    yield futs
    ex.shutdown(wait=True, cancel_futures=True)


def _gpu(args, kernel=lt.KERNEL_AUTO, layout=lt.INT8):
    dims, L, two_S, model, J, h, T, seed, init, n = args
    g = lt.Lattice(dims, L, two_S, model, J, h, T, seed=seed, init=init, layout=layout)
    try:
        if layout == lt.INT8:
            g.set_kernel(kernel, 0, 0, 0)
        g.sweep(n)
        spins, flags, done = g.get_state()
        assert done == n
        return spins, flags, g.series(0, n), g.get_kernel()
    finally:
        g.close()


def _compare(got, want, model):
    spins, flags, ser, _ = got
    ospins, oflags, oser = want
    bad = np.flatnonzero(spins != ospins)
    assert bad.size == 0, "spins differ at %d sites, first %s" % (bad.size, bad[:8])
    keys = ("bond", "mag", "up")
    if model == lt.NE:
        assert np.array_equal(flags, oflags), "persistence flags differ"
        keys += ("unflipped",)
    for k in keys:
        assert np.array_equal(ser[k], oser[k]), k


@pytest.mark.parametrize("T", TEMPS)
def test_L4096_int8_and_bitpacked_100_sweeps(oracle_runs, T):
    args = CASES[("ising", T)]
    runs = [_gpu(args)]                                         # autotuned, as the bench runs it
    runs += [_gpu(args, kernel=k) for k in (lt.KERNEL_WIDE, lt.KERNEL_TILED)]
    runs.append(_gpu(args, layout=lt.BITPACKED))
    want = oracle_runs[("ising", T)].result()
    for got in runs:
        _compare(got, want, lt.ISING)


def test_north_east_L8192_10_sweeps(oracle_runs):
    args = CASES[("ne", 0.3)]
    runs = [_gpu(args), _gpu(args, kernel=lt.KERNEL_TILED)]
    want = oracle_runs[("ne", 0.3)].result()
    for got in runs:
        _compare(got, want, lt.NE)


def test_3d_spin_one_L256_10_sweeps(oracle_runs):
    key = [k for k in CASES if k[0] == "3d"][0]
    args = CASES[key]
    runs = [_gpu(args), _gpu(args, kernel=lt.KERNEL_GENERIC)]
    want = oracle_runs[key].result()
    for got in runs:
        _compare(got, want, lt.ISING)
