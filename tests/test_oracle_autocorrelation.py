"""Pins of the oracle's spin-spin autocorrelation (CPU only).

§III.B defines Phi(t) from the overlap sum_i s_i(t) s_i(0) with the stored
initial configuration; the oracle records that overlap after every sweep.
It is pinned by cases whose value is fixed independently of the code:

* J = h = 0, spin-1/2: every spin flips every sweep (every move has
  dE = 0), so s(t) = (-1)^t s(0) and the overlap is (-1)^t N exactly, in
  2D and 3D.  A dropped colour, a wrong reference index or a sign slip
  breaks it.
* The overlap of a configuration with itself is sum_i s_i^2 (N for +-1
  spins, so Phi(0) = 1).
* J = h = 0, spin-1: every proposal is accepted and moves a site to one of
  its two other states with equal probability, so after one sweep
  E[s_i(1) s_i(0)] = -1/2 for s_i(0) = +-1 and 0 for s_i(0) = 0.
* North-East (§III.B): for c above the critical concentration Phi decays
  to zero; well below it most spins are stuck and Phi stays large.
"""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("dims,L", [(2, 8), (2, 14), (3, 6)])
def test_free_spins_alternate(dims, L):
    o = oracle.Lattice(dims, L, 1, oracle.ISING, 0.0, 0.0, 1.3, seed=5 + L, init=oracle.INIT_RANDOM)
    o.sweep(3)
    o.set_reference()
    ser = o.sweep(9)
    N = L ** dims
    assert list(ser["overlap"]) == [(-1) ** t * N for t in range(1, 10)]


@pytest.mark.parametrize("two_S", [1, 2, 3, 5])
def test_overlap_with_itself(two_S):
    o = oracle.Lattice(2, 10, two_S, oracle.ISING, 1.0, 0.0, 3.0, seed=9, init=oracle.INIT_RANDOM)
    o.sweep(2)
    o.set_reference()
    s = o.spins.astype(np.int64)
    assert o.overlap() == int((s * s).sum())
    if two_S == 1:
        assert o.overlap() == o.N


def test_spin_one_free_one_sweep_mean():
    # N = 64^2 sites, ~2/3 nonzero: C(1) has mean -nnz/2 and standard
    # deviation about sqrt(nnz)/2 (each term -1 or 0 with equal odds, or
    # 0 for s(0) = 0).  Accept within 5 standard deviations.
    o = oracle.Lattice(2, 64, 2, oracle.ISING, 0.0, 0.0, 1.0, seed=77, init=oracle.INIT_RANDOM)
    o.set_reference()
    nnz = int(np.count_nonzero(o.spins))
    c1 = int(o.sweep(1)["overlap"][0])
    sd = 0.5 * np.sqrt(nnz)
    assert abs(c1 + 0.5 * nnz) < 5 * sd, (c1, nnz)


def _phi(overlap, N, c):
    m = 2 * c - 1
    return (np.asarray(overlap, dtype=np.float64) / N - m * m) / (1 - m * m)


def test_north_east_phi_decays_above_critical_concentration():
    # c = 0.45 is above the critical concentration: Phi falls towards zero
    # (slowly under the facilitated rule: ~0.1 after 10^3 sweeps).
    o = oracle.Lattice(2, 48, 1, oracle.NE, 0.0, 0.0, 0.45, seed=21, init=oracle.INIT_EQUILIBRIUM)
    o.set_reference()
    phi = _phi(o.sweep(4000)["overlap"], o.N, 0.45)
    early, late = phi[100:200].mean(), phi[3500:].mean()
    assert abs(late) < 0.1
    assert late < 0.5 * early


def test_north_east_phi_stays_high_when_stuck():
    o = oracle.Lattice(2, 64, 1, oracle.NE, 0.0, 0.0, 0.05, seed=21, init=oracle.INIT_EQUILIBRIUM)
    o.set_reference()
    phi = _phi(o.sweep(300)["overlap"], o.N, 0.05)
    assert phi[-1] > 0.5
