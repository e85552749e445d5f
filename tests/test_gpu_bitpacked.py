"""Bit-packed spin-1/2 layout (one bit per site, one plane per colour):
bit for bit the same lattices and counters as the int8 layout and the CPU
oracle, since it uses the same Philox groups and thresholds.
"""
import numpy as np
import pytest

import oracle
import paper_1209_0296_gb300 as lt

pytestmark = pytest.mark.gpu


def _pair(L, model, J, h, Tc, seed, init, n):
    o = oracle.Lattice(2, L, 1, model, J, h, Tc, seed=seed, init=init)
    g = lt.Lattice(2, L, 1, model, J, h, Tc, seed=seed, init=init, layout=lt.BITPACKED)
    assert np.array_equal(g.get_spins(), o.spins)
    ser_o = o.sweep(n)
    g.sweep(n)
    spins, flags, done = g.get_state()
    assert done == n
    assert np.array_equal(spins, o.spins)
    if model == lt.NE:
        assert np.array_equal(flags, o.flags)
    ser = g.series(0, n)
    for k in ("bond", "mag", "up") + (("unflipped",) if model == lt.NE else ()):
        assert np.array_equal(ser[k], ser_o[k]), k
    return g


@pytest.mark.parametrize("L", [64, 128, 192])
@pytest.mark.parametrize("T,J,h", [(2.269185, 1.0, 0.0), (1.6, 1.0, 0.3), (3.2, -0.7, -0.2)])
def test_bitpacked_ising_matches_oracle(L, T, J, h):
    _pair(L, lt.ISING, J, h, T, 40 + L, lt.INIT_RANDOM, 30)


@pytest.mark.parametrize("c", [0.05, 0.3, 0.6])
def test_bitpacked_north_east_matches_oracle(c):
    _pair(128, lt.NE, 0.0, 0.0, c, 21, lt.INIT_EQUILIBRIUM, 40)


def test_bitpacked_equals_int8_long_run():
    a = lt.Lattice(2, 256, 1, lt.ISING, 1.0, 0.0, 2.269185, seed=7, init=lt.INIT_RANDOM)
    b = lt.Lattice(2, 256, 1, lt.ISING, 1.0, 0.0, 2.269185, seed=7, init=lt.INIT_RANDOM,
                   layout=lt.BITPACKED)
    a.sweep(500)
    b.sweep(500)
    assert np.array_equal(a.get_spins(), b.get_spins())
    for k in ("bond", "mag", "up"):
        assert np.array_equal(a.series()[k], b.series()[k])


def test_bitpacked_full_size_L4096():
    # 2D Ising spin-1/2, L=4096, T=2.0, random start (seed 7), bit-packed.
    _pair(4096, lt.ISING, 1.0, 0.0, 2.0, 7, lt.INIT_RANDOM, 3)


def test_bitpacked_checkpoint_and_unsupported():
    g = lt.Lattice(2, 64, 1, lt.NE, 0.0, 0.0, 0.4, seed=3, init=lt.INIT_EQUILIBRIUM,
                   layout=lt.BITPACKED)
    g.sweep(10)
    s, f, n = g.get_state()
    h = lt.Lattice(2, 64, 1, lt.NE, 0.0, 0.0, 0.4, seed=3, init=lt.INIT_EQUILIBRIUM,
                   layout=lt.BITPACKED)
    h.set_state(s, f, n)
    g.sweep(7)
    h.sweep(7)
    assert np.array_equal(g.get_state()[0], h.get_state()[0])
    assert np.array_equal(g.get_state()[1], h.get_state()[1])
    for bad in [dict(L=96, T_or_c=2.0), dict(L=64, T_or_c=0.3)]:
        with pytest.raises(lt.LatticeError) as e:
            lt.Lattice(2, bad["L"], 1, lt.ISING, 1.0, 0.0, bad["T_or_c"], seed=1, layout=lt.BITPACKED)
        assert e.value.code == -6
