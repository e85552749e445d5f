"""Pins of the oracle's q-state Potts model (the remark closing the paper's §III.A that
the method suits the Potts model; H = -J sum_<ij> delta(s_i, s_j) - h sum_i
delta(s_i, 0), labels 0..q-1, q = two_S + 1; CPU only).

* q = 2 is the Ising model: with sigma = 1 - 2s, the Potts chain at (J, h)
  is the Ising chain at (J/2, h/2) bit for bit -- same initial state, same
  draws, same thresholds -- and bond/mag map to 2*bond - (#bonds) and
  2*mag - N.
* J = h = 0: every proposal is accepted and goes to another state, so every
  site changes in every sweep.
* Exact averages: the 4x4 q = 3 (and q = 4) lattice by a transfer matrix over
  its rows, the 2x2x2 q = 3 lattice by brute force, against long runs.
* Baxter's critical point of the square lattice: at T_c = J / ln(1 + sqrt q)
  the energy per site is -J (1 + 1/sqrt q) (checked loosely at L = 64).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from tests.test_oracle_equilibrium import _mean_and_error


def _potts(dims, L, q, J, h, T, seed, init=oracle.INIT_RANDOM):
    return oracle.Lattice(dims, L, q - 1, oracle.POTTS, J, h, T, seed=seed, init=init)


@pytest.mark.parametrize("dims,L,h", [(2, 8, 0.0), (2, 10, 0.3), (3, 6, -0.2)])
@pytest.mark.parametrize("init", [oracle.INIT_RANDOM, oracle.INIT_COLD])
def test_q2_is_ising(dims, L, h, init):
    J, T = 1.3, 1.1
    p = _potts(dims, L, 2, J, h, T, 17, init)
    i = oracle.Lattice(dims, L, 1, oracle.ISING, J / 2, h / 2, T, seed=17, init=init)
    N = L ** dims
    assert np.array_equal(1 - 2 * p.spins.astype(np.int64), i.spins)
    for _ in range(4):
        sp, si = p.sweep(5), i.sweep(5)
        assert np.array_equal(1 - 2 * p.spins.astype(np.int64), i.spins)
        assert np.array_equal(2 * sp["bond"] - dims * N, si["bond"])
        assert np.array_equal(2 * sp["mag"] - N, si["mag"])


@pytest.mark.parametrize("q", [2, 3, 5, 9])
def test_free_labels_all_change(q):
    p = _potts(2, 8, q, 0.0, 0.0, 1.0, 4)
    for _ in range(5):
        before = p.spins.copy()
        p.sweep(1)
        assert np.all(p.spins != before)
        assert p.spins.min() >= 0 and p.spins.max() < q


def _lnZ_4x4(q, J, h, beta):
    rows = np.array(list(itertools.product(range(q), repeat=4)))
    e_row = -J * (rows == np.roll(rows, -1, axis=1)).sum(1) - h * (rows == 0).sum(1)
    e_int = -J * (rows[:, None, :] == rows[None, :, :]).sum(2)
    T = np.exp(-beta * (e_row[:, None] + e_int))
    return math.log(np.trace(np.linalg.matrix_power(T, 4)))


def _exact_4x4(q, J, h, temp):
    beta, d = 1.0 / temp, 1e-6
    E = -(_lnZ_4x4(q, J, h, beta + d) - _lnZ_4x4(q, J, h, beta - d)) / (2 * d) / 16
    n0 = (_lnZ_4x4(q, J, h + d, beta) - _lnZ_4x4(q, J, h - d, beta)) / (2 * d) / beta / 16
    return E, n0


@pytest.mark.parametrize("q,T,h", [(3, 1.0, 0.0), (3, 1.4, 0.3), (4, 0.9, 0.0)])
def test_enumeration_4x4(q, T, h):
    J = 1.0
    E, n0 = _exact_4x4(q, J, h, T)
    p = _potts(2, 4, q, J, h, T, 9)
    p.sweep(1000)
    ser = p.sweep(150000)
    e, de = _mean_and_error((-J * ser["bond"] - h * ser["mag"]) / 16)
    m, dm = _mean_and_error(ser["mag"] / 16)
    assert abs(e - E) < 5 * de + 1e-4, (e, E, de)
    assert abs(m - n0) < 5 * dm + 1e-4, (m, n0, dm)


def test_enumeration_3d_2x2x2():
    q, J, h, T = 3, 1.0, 0.2, 1.5
    states = np.array(list(itertools.product(range(q), repeat=8)))   # index x + 2y + 4z
    idx = np.arange(8)
    x, y, z = idx % 2, (idx // 2) % 2, idx // 4
    bond = np.zeros(len(states))
    for nb in (((x + 1) % 2) + 2 * y + 4 * z, x + 2 * ((y + 1) % 2) + 4 * z, x + 2 * y + 4 * ((z + 1) % 2)):
        bond += (states == states[:, nb]).sum(1)
    n0 = (states == 0).sum(1)
    E = -J * bond - h * n0
    w = np.exp(-(E - E.min()) / T)
    E_ex = (w * E).sum() / w.sum() / 8
    p = _potts(3, 2, q, J, h, T, 2)
    p.sweep(1000)
    ser = p.sweep(200000)
    e, de = _mean_and_error((-J * ser["bond"] - h * ser["mag"]) / 8)
    assert abs(e - E_ex) < 5 * de + 1e-4, (e, E_ex, de)


@pytest.mark.slow
def test_baxter_critical_energy():
    q, J = 3, 1.0
    Tc = J / math.log(1 + math.sqrt(q))
    p = _potts(2, 64, q, J, 0.0, Tc, 31)
    p.sweep(3000)
    ser = p.sweep(3000)
    u = (-J * ser["bond"] / 64 ** 2).mean()
    assert abs(u - (-J * (1 + 1 / math.sqrt(q)))) < 0.03, u


# The Potts overlap with a reference state is the number of sites whose label
# equals the reference label (the counterpart of Eq. 4's sum of s_i(t) s_i(0)).

@pytest.mark.parametrize("dims,L", [(2, 10), (3, 4)])
def test_overlap_q2_maps_to_the_ising_overlap(dims, L):
    # sigma = 1 - 2s: sum sigma sigma' = 2 * #equal - N, along the mapped chains
    J, h, T = 1.3, 0.2, 1.1
    p = _potts(dims, L, 2, J, h, T, 23)
    i = oracle.Lattice(dims, L, 1, oracle.ISING, J / 2, h / 2, T, seed=23, init=oracle.INIT_RANDOM)
    p.set_reference()
    i.set_reference()
    N = L ** dims
    sp, si = p.sweep(12), i.sweep(12)
    assert np.array_equal(2 * sp["overlap"] - N, si["overlap"])


@pytest.mark.parametrize("q", [3, 5])
def test_overlap_zero_temperature_moves(q):
    # J = h = 0: every site changes each sweep, so after one sweep no site
    # keeps its reference label; after two a site is back with chance
    # 1/(q-1) (the second move is uniform over the other q-1 labels)
    L, N = 16, 256
    p = _potts(2, L, q, 0.0, 0.0, 1.0, 5)
    p.set_reference()
    assert p.overlap() == N
    back = []
    for _ in range(300):
        p.set_reference()
        ser = p.sweep(2)
        assert ser["overlap"][0] == 0
        back.append(ser["overlap"][1])
    m, dm = _mean_and_error(np.array(back, dtype=np.float64))
    assert abs(m - N / (q - 1)) < 5 * dm, (m, dm)
