"""Pins of the oracle's update rule (CPU only).

* Acceptance thresholds vs Boltzmann weights: per-move detailed balance of
  the integer thresholds (§III.A: P_acc = min[1, exp(-dH/T)]), and the
  energy change against a brute-force energy difference of Eq. 2.
* One sweep, sampled many times by the oracle, against the exact per-site
  distribution computed from the paper's rule (tests/exact_small.py): this
  catches a wrong neighbour, sign, colour order, proposal or constraint.
* Special cases with closed-form outcomes: J = h = 0 flips every spin-1/2
  every sweep; a frozen cold lattice; the North-East all-up lattice becomes
  the deterministic checkerboard after one sweep at c < 1/2; all-down is
  absorbing (§III.B).
"""
import numpy as np
import pytest

import oracle
from tests import exact_small as ex


def _state_index(two_S, spins):
    vals = ex.spin_values(two_S)
    lut = {int(v): k for k, v in enumerate(vals)}
    return np.array([lut[int(s)] for s in spins])


@pytest.mark.parametrize("J,h,T", [(1.0, 0.0, 2.269185), (1.0, 0.3, 2.5), (-0.7, -0.5, 1.7),
                                   (0.4, 1.2, 0.9)])
@pytest.mark.parametrize("two_S", [1, 2, 3])
def test_threshold_detailed_balance(J, h, T, two_S):
    vals = ex.spin_values(two_S)
    zmax = 6 * int(vals.max())
    for s in vals:
        for s2 in vals:
            if s == s2:
                continue
            for n in range(-zmax, zmax + 1):
                dE = oracle.delta_energy(J, h, int(s2 - s), n)
                back = oracle.delta_energy(J, h, int(s - s2), n)
                assert dE == -back
                a_f, t_f = oracle.metropolis_threshold(dE, T)
                a_b, t_b = oracle.metropolis_threshold(back, T)
                A_f = 1.0 if a_f else t_f / 2.0**32
                A_b = 1.0 if a_b else t_b / 2.0**32
                # pi(s) A(s->s2) == pi(s2) A(s2->s), up to the 2^-32 quantisation
                # of each threshold (scaled by the Boltzmann ratio on the right).
                ratio = np.exp(-dE / T)
                assert abs(A_f - ratio * A_b) <= 2.0**-32 * (1.0 + ratio) * 1.000001
                assert a_f or a_b or dE == 0.0


@pytest.mark.parametrize("dims,L,two_S", [(2, 4, 1), (2, 4, 2), (3, 2, 1), (3, 2, 3)])
def test_delta_energy_matches_hamiltonian(dims, L, two_S):
    """dE of the oracle == H(after) - H(before) with H summed bond by bond (Eq. 2)."""
    rng = np.random.default_rng(3)
    vals = ex.spin_values(two_S)
    J, h = 0.8, -0.35
    bl = ex.bonds_forward(dims, L)
    nb = ex.neighbours(dims, L)

    def H(s):
        return -J * sum(int((s[a] * s[b]).sum()) for a, b in bl) - h * int(s.sum())

    for _ in range(40):
        s = vals[rng.integers(0, len(vals), L ** dims)]
        i = int(rng.integers(0, L ** dims))
        s2 = s.copy()
        s2[i] = vals[(list(vals).index(s[i]) + 1 + rng.integers(0, two_S)) % len(vals)]
        n = int(s[nb[i]].sum())
        dE = oracle.delta_energy(J, h, int(s2[i] - s[i]), n)
        assert dE == pytest.approx(H(s2) - H(s), abs=1e-12)


CASES = [
    # dims, L, two_S, model, J, h, T_or_c
    (2, 4, 1, oracle.ISING, 1.0, 0.3, 2.5),
    (2, 4, 1, oracle.ISING, -0.7, -0.5, 1.7),
    (2, 4, 2, oracle.ISING, 1.0, 0.2, 2.0),
    (3, 2, 1, oracle.ISING, 1.0, 0.1, 3.0),
    (3, 2, 3, oracle.ISING, 0.6, 0.0, 2.2),
    (2, 4, 1, oracle.NE, 0.0, 0.0, 0.3),
    (2, 4, 1, oracle.NE, 0.0, 0.0, 0.7),
    (2, 4, 1, oracle.NE, 0.5, -1.0, 1.5),
]


@pytest.mark.parametrize("case", CASES)
def test_one_sweep_distribution(case):
    dims, L, two_S, model, J, h, Tc = case
    rng = np.random.default_rng(11)
    vals = ex.spin_values(two_S)
    N = L ** dims
    k0 = rng.integers(0, len(vals), N)
    if model == oracle.NE:
        k0 = (rng.random(N) < 0.6).astype(np.int64)   # enough up spins to unlock moves
    P = ex.one_sweep_marginals(dims, L, two_S, model, J, h, Tc, k0)
    M = 12000
    counts = np.zeros_like(P)
    for seed in range(M):
        lat = oracle.Lattice(dims, L, two_S, model, J, h, Tc, seed=1000 + seed,
                             init=oracle.INIT_COLD)
        lat.spins[:] = vals[k0].astype(np.int8)
        lat.sweep(1)
        k1 = _state_index(two_S, lat.spins)
        counts[np.arange(N), k1] += 1
    emp = counts / M
    sigma = np.sqrt(np.maximum(P * (1 - P), 1.0 / M) / M)
    z = np.abs(emp - P) / sigma
    assert z.max() < 5.5, (z.max(), np.unravel_index(z.argmax(), z.shape))
    # Sites whose move is impossible must never move.
    assert np.all(emp[P == 0] == 0)


def test_zero_coupling_flips_every_spin_every_sweep():
    # J = h = 0: every dE = 0, so every proposal is accepted (§III.A rule).
    lat = oracle.Lattice(2, 10, 1, oracle.ISING, 0.0, 0.0, 1.3, seed=5, init=oracle.INIT_RANDOM)
    s0 = lat.spins.copy()
    for n in range(1, 6):
        lat.sweep(1)
        assert np.array_equal(lat.spins, s0 * (-1) ** n)
    lat3 = oracle.Lattice(3, 4, 2, oracle.ISING, 0.0, 0.0, 1.0, seed=6, init=oracle.INIT_RANDOM)
    prev = lat3.spins.copy()
    lat3.sweep(1)
    assert np.all(lat3.spins != prev)


@pytest.mark.parametrize("dims,L,two_S", [(2, 8, 1), (3, 4, 1), (2, 6, 2)])
def test_cold_lattice_frozen_at_low_temperature(dims, L, two_S):
    lat = oracle.Lattice(dims, L, two_S, oracle.ISING, 1.0, 0.0, 1e-3, seed=9, init=oracle.INIT_COLD)
    top = int(ex.spin_values(two_S).max())
    ser = lat.sweep(4)
    N = L ** dims
    assert np.all(lat.spins == top)
    assert np.all(ser["bond"] == dims * N * top * top)
    assert np.all(ser["mag"] == N * top)


def test_north_east_all_up_becomes_checkerboard():
    # c < 1/2: up->down is always accepted; from all-up, every colour-0 site
    # is unlocked and flips down, after which no colour-1 site is unlocked.
    for seed in (1, 2, 3):
        lat = oracle.Lattice(2, 8, 1, oracle.NE, 0.0, 0.0, 0.2, seed=seed, init=oracle.INIT_COLD)
        ser = lat.sweep(1)
        x, y, _ = ex.coords(2, 8)
        expect = np.where((x + y) % 2 == 0, -1, 1)
        assert np.array_equal(lat.spins, expect)
        assert ser["up"][0] == 32 and ser["unflipped"][0] == 32


def test_north_east_all_down_is_absorbing():
    lat = oracle.Lattice(2, 8, 1, oracle.NE, 0.0, 0.0, 0.3, seed=4, init=oracle.INIT_COLD)
    lat.spins[:] = -1
    ser = lat.sweep(5)
    assert np.all(lat.spins == -1)
    assert np.all(ser["up"] == 0) and np.all(ser["unflipped"] == 64)


def test_north_east_constraint_and_persistence_invariants():
    L = 16
    lat = oracle.Lattice(2, L, 1, oracle.NE, 0.0, 0.0, 0.35, seed=21, init=oracle.INIT_EQUILIBRIUM)
    x, y, _ = ex.coords(2, L)
    colour = (x + y) % 2
    north = ex.index(2, L, x, y - 1, 0)
    east = ex.index(2, L, x + 1, y, 0)
    s_init = lat.spins.copy()
    ever = np.zeros(L * L, dtype=bool)
    last_unflipped = L * L
    moved = 0
    for _ in range(30):
        before = lat.spins.copy()
        ser = lat.sweep(1)
        after = lat.spins.copy()
        ch = before != after
        moved += ch.sum()
        # colour-0 sites move first: their north/east (colour 1) are as before.
        c0 = ch & (colour == 0)
        assert np.all(before[north[c0]] == 1) and np.all(before[east[c0]] == 1)
        # colour-1 sites move second: their north/east (colour 0) are as after.
        c1 = ch & (colour == 1)
        assert np.all(after[north[c1]] == 1) and np.all(after[east[c1]] == 1)
        ever |= ch
        assert np.array_equal(lat.flags.astype(bool), ever)
        assert ser["unflipped"][0] <= last_unflipped
        last_unflipped = ser["unflipped"][0]
        assert ser["up"][0] == int((after == 1).sum())
    assert moved > 0
    # A site whose flag is clear still holds its initial value.
    assert np.all(lat.spins[lat.flags == 0] == s_init[lat.flags == 0])


def test_spin_values_stay_in_allowed_set():
    for two_S in (1, 2, 3, 4):
        lat = oracle.Lattice(2, 6, two_S, oracle.ISING, 1.0, 0.2, 2.0, seed=two_S,
                             init=oracle.INIT_RANDOM)
        lat.sweep(10)
        assert set(np.unique(lat.spins)).issubset(set(ex.spin_values(two_S).tolist()))


def test_series_match_final_lattice():
    lat = oracle.Lattice(3, 4, 2, oracle.ISING, 1.0, 0.0, 3.0, seed=8, init=oracle.INIT_RANDOM)
    ser = lat.sweep(3)
    s = lat.spins.astype(np.int64)
    bond = sum(int((s[a] * s[b]).sum()) for a, b in ex.bonds_forward(3, 4))
    assert ser["bond"][-1] == bond
    assert ser["mag"][-1] == s.sum()
    assert ser["up"][-1] == (s > 0).sum()


def test_invalid_parameters_rejected():
    for args in [(2, 5, 1, 0, 1.0, 0.0, 2.0), (4, 4, 1, 0, 1.0, 0.0, 2.0),
                 (3, 4, 1, 1, 0.0, 0.0, 0.3), (2, 4, 2, 1, 0.0, 0.0, 0.3),
                 (2, 4, 1, 1, 0.0, 0.0, 1.5), (2, 4, 1, 0, 1.0, 0.0, -1.0),
                 (2, 4, 0, 0, 1.0, 0.0, 2.0)]:
        with pytest.raises(ValueError):
            oracle.Lattice(*args)
