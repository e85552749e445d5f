"""Pins of the oracle's random-sub-lattice, random-site North-East algorithm
(§III.B, the paper's own GPU algorithm; CPU only).

* Closed form, J = h = 0 (every move allowed and accepted): a site changes
  once per round in which it is picked at least once, so after one sweep
  (P/lambda rounds per sub-lattice) E[s_i(1) s_i(0)] = (1 - 2 pi)^(P/lambda)
  with pi = 1 - (1 - 1/P)^lambda.  This fixes the uniform pick, the number of
  rounds and the rule that simultaneous picks of a site change it once.
* The serial limit Q = lambda = 1 (one sub-lattice, one pick per round) is
  random-site Metropolis, which keeps detailed balance: its long-run
  averages equal Boltzmann enumeration (4x4 Ising) and the North-East
  density equals c.
* §III.B, Fig. 5: with small lambda (16 picks per 32x32 sub-lattice) the
  relaxation Phi(t) follows the serial one; with lambda = P/2 it departs.
* The North-East all-down state is absorbing for any sub-lattice and lambda.

The balance-preserving variant (single-colour rounds, four launches):
* Closed form, J = h = 0: a site is picked in a round of its colour with
  chance pi' = 1 - (1 - 2/P)^lambda and meets q = P/(2 lambda) such rounds
  per sweep, so E[s_i(1) s_i(0)] = (1 - 2 pi')^q.
* With one sub-lattice its rounds change only non-interacting sites, so
  Boltzmann averages hold for lambda > 1 (4x4 enumeration), where the plain
  algorithm's concurrent picks are measurably off (the paper: the plain
  algorithm keeps neither detailed nor the weaker balance).
"""
import math

import numpy as np
import pytest

import oracle
from tests import exact_small as ex
from tests.test_oracle_equilibrium import _mean_and_error


def _overlap_after_one_sweep(L, b, lam, seed):
    o = oracle.Lattice(2, L, 1, oracle.ISING, 0.0, 0.0, 1.0, seed=seed, init=oracle.INIT_RANDOM)
    o.set_reference()
    return o.rsite_sweep(1, b, lam)["overlap"][0] / o.N


@pytest.mark.parametrize("L,b,lam", [(64, 64, 1), (64, 64, 2048), (64, 16, 1), (64, 16, 8),
                                     (64, 8, 32), (32, 32, 512)])
def test_free_spins_one_sweep_closed_form(L, b, lam):
    P = b * b
    pi = 1.0 - (1.0 - 1.0 / P) ** lam
    expect = (1.0 - 2.0 * pi) ** (P // lam)
    runs = [_overlap_after_one_sweep(L, b, lam, seed) for seed in range(12)]
    # each site's sign is an independent +-1 with mean `expect`
    sd = math.sqrt((1.0 - expect ** 2) / (L * L) / len(runs))
    assert abs(np.mean(runs) - expect) < 5 * sd + 1e-3, (np.mean(runs), expect, sd)


@pytest.mark.parametrize("T", [2.0, 3.0])
def test_serial_limit_matches_enumeration(T):
    E, M, _ = ex.enumerate_averages(2, 4, 1, 1.0, 0.0, T)
    o = oracle.Lattice(2, 4, 1, oracle.ISING, 1.0, 0.0, T, seed=5, init=oracle.INIT_RANDOM)
    o.rsite_sweep(500, 4, 1)
    ser = o.rsite_sweep(100000, 4, 1)
    e, de = _mean_and_error(o.energy(ser["bond"], ser["mag"]) / 16)
    m, dm = _mean_and_error(np.abs(ser["mag"]) / 16)
    assert abs(e - E) < 5 * de + 1e-4, (e, E, de)
    assert abs(m - M) < 5 * dm + 1e-4, (m, M, dm)


@pytest.mark.parametrize("c", [0.2, 0.42])
def test_serial_limit_north_east_density(c):
    # From an equilibrium sample the serial dynamics keeps the density at c
    # up to that sample's own noise (frozen clusters on a finite torus keep
    # the time average from converging to c itself).
    L = 64
    o = oracle.Lattice(2, L, 1, oracle.NE, 0.0, 0.0, c, seed=7, init=oracle.INIT_EQUILIBRIUM)
    ser = o.rsite_sweep(400, L, 1)
    assert abs((ser["up"] / (L * L)).mean() - c) < 5 * math.sqrt(c * (1 - c) / (L * L))


def test_serial_limit_north_east_relaxes_to_c():
    # from all-up at c = 0.45 (well above c*), the serial dynamics relaxes to
    # density c, the only stationary density of the c-mode rates
    c, L = 0.45, 32
    o = oracle.Lattice(2, L, 1, oracle.NE, 0.0, 0.0, c, seed=33, init=oracle.INIT_COLD)
    o.rsite_sweep(300, L, 1)
    ser = o.rsite_sweep(4000, L, 1)
    rho, err = _mean_and_error(ser["up"] / (L * L))
    assert abs(rho - c) < 5 * err + 2e-3, (rho, err)


def _phi_curve(L, b, lam, seeds, n, c=0.42):
    m = 2 * c - 1
    acc = np.zeros(n)
    for seed in seeds:
        o = oracle.Lattice(2, L, 1, oracle.NE, 0.0, 0.0, c, seed=seed, init=oracle.INIT_EQUILIBRIUM)
        o.set_reference()
        ov = o.rsite_sweep(n, b, lam)["overlap"]
        acc += (ov / o.N - m * m) / (1 - m * m)
    return acc / len(seeds)


@pytest.mark.slow
def test_small_lambda_follows_the_serial_relaxation():
    # c = 0.42 as in Fig. 5; L = 64 so the serial reference is one 64x64
    # sub-lattice with one pick per round
    n, seeds = 30, range(6)
    serial = _phi_curve(64, 64, 1, seeds, n)
    small = _phi_curve(64, 32, 16, seeds, n)
    large = _phi_curve(64, 32, 512, seeds, n)
    d_small = np.abs(small - serial).mean()
    d_large = np.abs(large - serial).mean()
    assert d_small < 0.03, d_small
    assert d_large > 2 * d_small, (d_small, d_large)


@pytest.mark.parametrize("b,lam", [(8, 4), (16, 128)])
def test_all_down_is_absorbing(b, lam):
    o = oracle.Lattice(2, 32, 1, oracle.NE, 0.0, 0.0, 0.3, seed=1, init=oracle.INIT_COLD)
    o.spins[:] = -1
    ser = o.rsite_sweep(5, b, lam)
    assert (o.spins == -1).all()
    assert list(ser["up"]) == [0] * 5


# ---- the balance-preserving variant -------------------------------------

def _balanced_overlap_after_one_sweep(L, b, lam, seed):
    o = oracle.Lattice(2, L, 1, oracle.ISING, 0.0, 0.0, 1.0, seed=seed, init=oracle.INIT_RANDOM)
    o.set_reference()
    return o.rsite_sweep(1, b, lam, balanced=True)["overlap"][0] / o.N


@pytest.mark.parametrize("L,b,lam", [(64, 64, 1), (64, 16, 8), (64, 8, 4), (32, 32, 64), (64, 64, 512)])
def test_balanced_free_spins_one_sweep_closed_form(L, b, lam):
    P = b * b
    q = P // (2 * lam)
    pi = 1.0 - (1.0 - 2.0 / P) ** lam
    expect = (1.0 - 2.0 * pi) ** q
    runs = [_balanced_overlap_after_one_sweep(L, b, lam, seed) for seed in range(12)]
    sd = math.sqrt((1.0 - expect ** 2) / (L * L) / len(runs))
    assert abs(np.mean(runs) - expect) < 5 * sd + 1e-3, (np.mean(runs), expect, sd)


@pytest.mark.parametrize("T", [2.0, 3.0])
def test_balanced_one_sublattice_keeps_boltzmann(T):
    E, M, _ = ex.enumerate_averages(2, 4, 1, 1.0, 0.0, T)
    o = oracle.Lattice(2, 4, 1, oracle.ISING, 1.0, 0.0, T, seed=5, init=oracle.INIT_RANDOM)
    o.rsite_sweep(500, 4, 2, balanced=True)
    ser = o.rsite_sweep(100000, 4, 2, balanced=True)
    e, de = _mean_and_error(o.energy(ser["bond"], ser["mag"]) / 16)
    m, dm = _mean_and_error(np.abs(ser["mag"]) / 16)
    assert abs(e - E) < 5 * de + 1e-4, (e, E, de)
    assert abs(m - M) < 5 * dm + 1e-4, (m, M, dm)


def test_plain_concurrent_picks_break_balance():
    # the same lattice, sub-lattice and lambda with the plain algorithm
    T = 3.0
    E, _, _ = ex.enumerate_averages(2, 4, 1, 1.0, 0.0, T)
    o = oracle.Lattice(2, 4, 1, oracle.ISING, 1.0, 0.0, T, seed=5, init=oracle.INIT_RANDOM)
    o.rsite_sweep(500, 4, 2)
    ser = o.rsite_sweep(100000, 4, 2)
    e, de = _mean_and_error(o.energy(ser["bond"], ser["mag"]) / 16)
    assert abs(e - E) > 5 * de, (e, E, de)


def test_balanced_north_east_density():
    c, L = 0.3, 32
    o = oracle.Lattice(2, L, 1, oracle.NE, 0.0, 0.0, c, seed=9, init=oracle.INIT_EQUILIBRIUM)
    ser = o.rsite_sweep(300, L, 4, balanced=True)
    assert abs((ser["up"] / (L * L)).mean() - c) < 5 * math.sqrt(c * (1 - c) / (L * L))
    o.spins[:] = -1
    ser = o.rsite_sweep(3, 8, 4, balanced=True)
    assert (o.spins == -1).all() and list(ser["up"]) == [0] * 3


def test_balanced_needs_q_multiple_of_four():
    o = oracle.Lattice(2, 16, 1, oracle.ISING, 1.0, 0.0, 2.0, seed=1, init=oracle.INIT_RANDOM)
    with pytest.raises(ValueError):
        o.rsite_sweep(1, 8, 16, balanced=True)   # q = 32/16 = 2
