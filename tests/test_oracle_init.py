"""Pins for the oracle's initial states (oracle_init).

§III.A step 1 starts from a random lattice and §III.B step 1 puts each
site up with probability c (the North-East model's equilibrium).  The
checks below are what those definitions fix, independent of how the
oracle draws:
  - a cold start is exactly the top state everywhere;
  - a random spin-1/2 start is up with probability 1/2, a spin-S start is
    uniform over the 2S+1 states and a q-state Potts start uniform over
    the q labels (each within 5 sigma on 2^18 sites);
  - an equilibrium start is up with probability c (5 sigma);
  - sites are independent: the four sites that share one Philox call and
    neighbouring sites show no correlation beyond 5 sigma;
  - two starts that the definitions make identical are identical bit for
    bit: the equilibrium start at c = 1/2 and the random spin-1/2 start
    (both "up with probability 1/2"), and the Potts q = 2 start and the
    Ising start through label 0 <-> up;
  - the initial state depends on the seed alone (not on T or the model
    parameters) and on all 64 bits of it.
"""
import math

import numpy as np
import pytest

import oracle

N2 = 512          # 2D side: 2^18 sites
N3 = 64           # 3D side: 2^18 sites


def _frac_ok(count, n, p, k=5.0):
    sd = math.sqrt(p * (1.0 - p) / n)
    return abs(count / n - p) <= k * sd, (count / n, p, sd)


def _spin_values(two_S):
    return [(2 * k - two_S) if two_S & 1 else (k - two_S // 2) for k in range(two_S + 1)]


@pytest.mark.parametrize("dims,L", [(2, N2), (3, N3)])
@pytest.mark.parametrize("two_S", [1, 2, 3, 4])
def test_cold_start_is_all_top(dims, L, two_S):
    lat = oracle.Lattice(dims, L, two_S, oracle.ISING, 1.0, 0.0, 2.0, seed=3, init=oracle.INIT_COLD)
    top = _spin_values(two_S)[-1]
    assert np.all(lat.spins == top)


@pytest.mark.parametrize("q", [2, 3, 4])
def test_potts_cold_start_is_label_zero(q):
    lat = oracle.Lattice(2, 64, q - 1, oracle.POTTS, 1.0, 0.0, 1.0, seed=3, init=oracle.INIT_COLD)
    assert np.all(lat.spins == 0)


@pytest.mark.parametrize("dims,L", [(2, N2), (3, N3)])
def test_random_spin_half_is_fair_and_independent(dims, L):
    lat = oracle.Lattice(dims, L, 1, oracle.ISING, 1.0, 0.0, 3.0, seed=7, init=oracle.INIT_RANDOM)
    s = lat.spins
    n = s.size
    assert set(np.unique(s).tolist()) == {-1, 1}
    up = s > 0
    ok, info = _frac_ok(int(up.sum()), n, 0.5)
    assert ok, info
    # each of the four words of a Philox call is fair on its own
    for q in range(4):
        ok, info = _frac_ok(int(up[q::4].sum()), n // 4, 0.5)
        assert ok, (q, info)
    # pairs inside one call, and across neighbouring calls, are independent:
    # P(both up) = 1/4 (a word reused for two sites would give 1/2)
    g = up.reshape(-1, 4)
    for a in range(4):
        for b in range(a + 1, 4):
            ok, info = _frac_ok(int((g[:, a] & g[:, b]).sum()), g.shape[0], 0.25)
            assert ok, (a, b, info)
    for q in range(4):
        ok, info = _frac_ok(int((g[:-1, q] & g[1:, q]).sum()), g.shape[0] - 1, 0.25)
        assert ok, (q, info)
    # lattice neighbours along y (and z) are independent too
    sl = up.reshape((L,) * dims)
    ok, info = _frac_ok(int((sl & np.roll(sl, 1, axis=0)).sum()), n, 0.25)
    assert ok, info


@pytest.mark.parametrize("dims,L", [(2, N2), (3, N3)])
@pytest.mark.parametrize("two_S", [2, 3, 4])
def test_random_spin_S_is_uniform_over_the_states(dims, L, two_S):
    lat = oracle.Lattice(dims, L, two_S, oracle.ISING, 1.0, 0.0, 3.0, seed=11, init=oracle.INIT_RANDOM)
    s = lat.spins
    vals = _spin_values(two_S)
    assert set(np.unique(s).tolist()) <= set(vals)
    for v in vals:     # every state, the top one included, has weight 1/(2S+1)
        ok, info = _frac_ok(int((s == v).sum()), s.size, 1.0 / (two_S + 1))
        assert ok, (v, info)


@pytest.mark.parametrize("q", [2, 3, 4, 5])
def test_random_potts_is_uniform_over_the_labels(q):
    lat = oracle.Lattice(2, N2, q - 1, oracle.POTTS, 1.0, 0.0, 1.0, seed=13, init=oracle.INIT_RANDOM)
    s = lat.spins
    assert set(np.unique(s).tolist()) <= set(range(q))
    for k in range(q):
        ok, info = _frac_ok(int((s == k).sum()), s.size, 1.0 / q)
        assert ok, (k, info)


@pytest.mark.parametrize("c", [0.05, 0.1, 0.3, 0.45])
def test_equilibrium_start_is_up_with_probability_c(c):
    lat = oracle.Lattice(2, N2, 1, oracle.NE, 0.0, 0.0, c, seed=21, init=oracle.INIT_EQUILIBRIUM)
    s = lat.spins
    assert set(np.unique(s).tolist()) <= {-1, 1}
    ok, info = _frac_ok(int((s > 0).sum()), s.size, c)
    assert ok, info
    # independent sites: P(site and its north neighbour both up) = c^2
    up = (s > 0).reshape(N2, N2)
    ok, info = _frac_ok(int((up & np.roll(up, 1, axis=0)).sum()), s.size, c * c)
    assert ok, info


def test_equilibrium_at_one_half_is_the_random_start():
    # "up with probability c" at c = 1/2 is "up with probability 1/2"
    a = oracle.Lattice(2, 256, 1, oracle.NE, 0.0, 0.0, 0.5, seed=5, init=oracle.INIT_EQUILIBRIUM)
    b = oracle.Lattice(2, 256, 1, oracle.ISING, 1.0, 0.0, 2.0, seed=5, init=oracle.INIT_RANDOM)
    assert np.array_equal(a.spins, b.spins)


def test_equilibrium_density_grows_with_c():
    # the same draws at a larger c can only add up sites (u < thr_c is monotone in c)
    lo = oracle.Lattice(2, 256, 1, oracle.NE, 0.0, 0.0, 0.1, seed=5, init=oracle.INIT_EQUILIBRIUM).spins
    hi = oracle.Lattice(2, 256, 1, oracle.NE, 0.0, 0.0, 0.3, seed=5, init=oracle.INIT_EQUILIBRIUM).spins
    assert np.all(hi[lo > 0] > 0)
    assert (hi > 0).sum() > (lo > 0).sum()


def test_potts_q2_start_is_the_ising_start():
    # Potts q = 2 is Ising with label 0 <-> up (sigma = 1 - 2 s)
    p = oracle.Lattice(2, 256, 1, oracle.POTTS, 1.0, 0.0, 1.0, seed=9, init=oracle.INIT_RANDOM).spins
    i = oracle.Lattice(2, 256, 1, oracle.ISING, 1.0, 0.0, 2.0, seed=9, init=oracle.INIT_RANDOM).spins
    assert np.array_equal(1 - 2 * p.astype(np.int64), i.astype(np.int64))


def test_start_depends_on_the_seed_only():
    base = oracle.Lattice(2, 128, 1, oracle.ISING, 1.0, 0.0, 2.0, seed=7, init=oracle.INIT_RANDOM).spins
    # temperature, coupling and field do not enter the initial state
    for T, J, h in [(3.0, 1.0, 0.0), (1.0, -1.0, 0.5)]:
        other = oracle.Lattice(2, 128, 1, oracle.ISING, J, h, T, seed=7, init=oracle.INIT_RANDOM).spins
        assert np.array_equal(base, other)
    # every bit of the 64-bit seed matters: lo word, hi word
    for seed in (8, 7 + (1 << 32), 7 + (1 << 63)):
        other = oracle.Lattice(2, 128, 1, oracle.ISING, 1.0, 0.0, 2.0, seed=seed, init=oracle.INIT_RANDOM).spins
        diff = np.mean(base != other)
        assert 0.45 < diff < 0.55, (seed, diff)
