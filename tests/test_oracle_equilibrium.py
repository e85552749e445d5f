"""Equilibrium pins of the oracle (CPU only).

The paper validates its sweeps by the thermodynamics they reach (§V.A, Fig. 3:
magnetisation, energy and heat capacity against a CPU code) and relies on the
sweep keeping balance (§III.A).  Here the oracle's long-run averages are held
against results that do not come from any sweep:

* exact Boltzmann averages by enumeration of every configuration of tiny
  periodic lattices (spin-1/2 and spin-1, 2D and 3D);
* Onsager's closed form for the 2D Ising internal energy and Yang's
  spontaneous magnetisation (the paper quotes T_c = 2/log(1+sqrt 2), §V.A);
* the North-East model's uncorrelated equilibrium: up density = c (§III.B).
"""
import math

import numpy as np
import pytest
from scipy.special import ellipk

import oracle
from tests import exact_small as ex


def _mean_and_error(x, nblocks=40):
    """Mean with a blocking (batch-means) standard error."""
    x = np.asarray(x, dtype=np.float64)
    n = (x.size // nblocks) * nblocks
    blocks = x[:n].reshape(nblocks, -1).mean(axis=1)
    return x[:n].mean(), blocks.std(ddof=1) / math.sqrt(nblocks)


def _run_averages(dims, L, two_S, J, h, T, sweeps, burn, seed, init=oracle.INIT_RANDOM):
    lat = oracle.Lattice(dims, L, two_S, oracle.ISING, J, h, T, seed=seed, init=init)
    lat.sweep(burn)
    ser = lat.sweep(sweeps)
    N = L ** dims
    e = lat.energy(ser["bond"], ser["mag"]) / N
    m = np.abs(ser["mag"]) / N
    return _mean_and_error(e), _mean_and_error(m), _mean_and_error((ser["mag"] / N) ** 2)


@pytest.mark.parametrize("L,two_S,J,h,T", [(4, 1, 1.0, 0.2, 2.3), (2, 2, 0.7, 0.1, 1.5),
                                           (2, 3, -0.5, 0.3, 4.0)])
def test_row_and_site_enumerations_agree(L, two_S, J, h, T):
    a = ex.enumerate_averages(2, L, two_S, J, h, T)
    b = ex.enumerate_sites(2, L, two_S, J, h, T)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("T", [2.0, 2.269185, 3.0])
def test_enumeration_2d_spin_half_4x4(T):
    E, M, _ = ex.enumerate_averages(2, 4, 1, 1.0, 0.0, T)
    (e, de), (m, dm), _ = _run_averages(2, 4, 1, 1.0, 0.0, T, 200000, 1000, seed=17)
    assert abs(e - E) < 5 * de + 1e-4, (e, E, de)
    assert abs(m - M) < 5 * dm + 1e-4, (m, M, dm)


def test_enumeration_2d_spin_half_field():
    E, M, M2 = ex.enumerate_averages(2, 4, 1, 0.7, 0.25, 2.4)
    (e, de), _, (m2, dm2) = _run_averages(2, 4, 1, 0.7, 0.25, 2.4, 150000, 1000, seed=18)
    assert abs(e - E) < 5 * de + 1e-4
    assert abs(m2 - M2) < 5 * dm2 + 1e-4


@pytest.mark.parametrize("two_S,T", [(1, 4.5), (2, 3.0), (3, 30.0)])
def test_enumeration_3d_L2(two_S, T):
    E, M, M2 = ex.enumerate_averages(3, 2, two_S, 1.0, 0.1, T)
    (e, de), (m, dm), (m2, dm2) = _run_averages(3, 2, two_S, 1.0, 0.1, T, 150000, 1000,
                                               seed=19)
    assert abs(e - E) < 5 * de + 1e-4, (e, E, de)
    assert abs(m - M) < 5 * dm + 1e-4, (m, M, dm)
    assert abs(m2 - M2) < 5 * dm2 + 1e-4


def test_enumeration_2d_spin_one_4x4():
    # 3^16 = 43,046,721 configurations, enumerated row by row.
    E, M, M2 = ex.enumerate_averages(2, 4, 2, 1.0, 0.0, 1.6)
    (e, de), (m, dm), _ = _run_averages(2, 4, 2, 1.0, 0.0, 1.6, 150000, 1000, seed=20)
    assert abs(e - E) < 5 * de + 1e-4, (e, E, de)
    assert abs(m - M) < 5 * dm + 1e-4, (m, M, dm)


def onsager_energy(T, J=1.0):
    """Onsager's internal energy per site of the infinite 2D Ising model."""
    b = 1.0 / T
    k = 2.0 * math.sinh(2 * b * J) / math.cosh(2 * b * J) ** 2
    K = ellipk(k * k)
    return -J / math.tanh(2 * b * J) * (1 + 2 / math.pi * (2 * math.tanh(2 * b * J) ** 2 - 1) * K)


def yang_magnetisation(T, J=1.0):
    s = math.sinh(2 * J / T)
    return (1 - s ** -4) ** 0.125 if s > 1 else 0.0


def test_onsager_closed_forms_themselves():
    # u(T_c) = -sqrt(2) and m vanishes at T_c = 2/log(1+sqrt 2) (§V.A).
    Tc = 2 / math.log(1 + math.sqrt(2))
    # (K diverges at T_c itself while its prefactor vanishes: take the limit.)
    assert onsager_energy(Tc * (1 + 1e-7)) == pytest.approx(-math.sqrt(2), abs=1e-5)
    assert onsager_energy(Tc * (1 - 1e-7)) == pytest.approx(-math.sqrt(2), abs=1e-5)
    assert yang_magnetisation(Tc * (1 + 1e-9)) == 0.0
    assert onsager_energy(2.0) == pytest.approx(-1.745565, abs=2e-6)
    assert yang_magnetisation(2.0) == pytest.approx(0.911319, abs=2e-6)


@pytest.mark.slow
def test_onsager_ordered_phase_cold_start():
    (e, de), (m, dm), _ = _run_averages(2, 128, 1, 1.0, 0.0, 2.0, 2400, 400, seed=23,
                                        init=oracle.INIT_COLD)
    assert abs(e - onsager_energy(2.0)) < 5 * de + 2e-4, (e, de)
    assert abs(m - yang_magnetisation(2.0)) < 5 * dm + 2e-4, (m, dm)


@pytest.mark.slow
def test_onsager_disordered_phase_random_start():
    (e, de), (m, dm), _ = _run_averages(2, 128, 1, 1.0, 0.0, 3.0, 2400, 400, seed=24)
    assert abs(e - onsager_energy(3.0)) < 5 * de + 2e-4, (e, de)
    assert m < 0.05


@pytest.mark.parametrize("c", [0.1, 0.3, 0.45])
def test_north_east_density_equals_c(c):
    L = 64
    lat = oracle.Lattice(2, L, 1, oracle.NE, 0.0, 0.0, c, seed=31, init=oracle.INIT_EQUILIBRIUM)
    ser = lat.sweep(1500)
    rho = ser["up"] / (L * L)
    # A fresh equilibrium lattice already has density c up to its own
    # sampling noise; the dynamics must keep it there (stationarity).
    assert abs(rho.mean() - c) < 5 * math.sqrt(c * (1 - c) / (L * L))
    # and the persistence is non-increasing and in [0, 1].
    P = ser["unflipped"] / (L * L)
    assert np.all(np.diff(P) <= 0) and 0 <= P[-1] <= 1


def test_north_east_density_from_far_start():
    # From all-up, the density relaxes to c (the only stationary density of
    # the unconstrained c-mode rates, §III.B) when c is well above c* ~ 0.3.
    c, L = 0.45, 32
    lat = oracle.Lattice(2, L, 1, oracle.NE, 0.0, 0.0, c, seed=33, init=oracle.INIT_COLD)
    lat.sweep(300)
    ser = lat.sweep(6000)
    rho, err = _mean_and_error(ser["up"] / (L * L))
    assert abs(rho - c) < 5 * err + 2e-3, (rho, err)
