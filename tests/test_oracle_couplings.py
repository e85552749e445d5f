"""Pins of the oracle's per-bond couplings (Eq. 1: J_ij = J * eps_ij with
eps_ij = +-1, nearest neighbours; the Edwards-Anderson +-J spin glass;
CPU only).

* Gauge invariance: with tau_i = +-1, the couplings eps'_ij = tau_i tau_j
  eps_ij and the start tau*s(0) give every move the same energy change, so
  with the same random numbers the chain is tau*s(t) at every sweep and the
  weighted bond sums are equal (spin-1/2, h = 0: the flip is symmetric).  A
  bond read from the wrong site or direction breaks this.
* All eps = +1 is the ferromagnet and all eps = -1 the J -> -J model: the
  chains equal the oracle's uniform-coupling chains bit for bit.
* Boltzmann enumeration of a random 4x4 instance in a field.
"""
import math

import numpy as np
import pytest

import oracle
from tests.test_oracle_equilibrium import _mean_and_error


def _lat(dims, L, two_S, J, h, T, seed, eps=None, spins=None):
    o = oracle.Lattice(dims, L, two_S, oracle.ISING, J, h, T, seed=seed, init=oracle.INIT_RANDOM)
    if spins is not None:
        o.spins[:] = spins
    o.set_couplings(eps)
    return o


def _gauge(dims, L, eps, tau):
    N = L ** dims
    idx = np.arange(N)
    coords = [(idx // L ** d) % L for d in range(dims)]
    out = eps.copy().reshape(dims, N)
    for d in range(dims):
        nb = coords.copy()
        nb[d] = (coords[d] + 1) % L
        j = sum(nb[k] * L ** k for k in range(dims))
        out[d] = out[d] * tau * tau[j]
    return out.reshape(-1)


@pytest.mark.parametrize("dims,L", [(2, 8), (2, 10), (3, 6)])
def test_gauge_invariance(dims, L):
    rng = np.random.default_rng(L + dims)
    N = L ** dims
    eps = rng.choice(np.array([-1, 1], dtype=np.int8), dims * N)
    tau = rng.choice(np.array([-1, 1], dtype=np.int8), N)
    a = _lat(dims, L, 1, 1.0, 0.0, 1.6, 21, eps)
    b = _lat(dims, L, 1, 1.0, 0.0, 1.6, 21, _gauge(dims, L, eps, tau), spins=a.spins * tau)
    for _ in range(6):
        sa, sb = a.sweep(3), b.sweep(3)
        assert np.array_equal(b.spins, a.spins * tau)
        assert np.array_equal(sa["bond"], sb["bond"])


@pytest.mark.parametrize("dims,L,two_S", [(2, 8, 1), (3, 6, 1), (2, 6, 2), (3, 4, 3)])
@pytest.mark.parametrize("sign", [1, -1])
def test_uniform_couplings_reduce_to_the_plain_model(dims, L, two_S, sign):
    N = L ** dims
    eps = np.full(dims * N, sign, dtype=np.int8)
    T = 2.0 * two_S
    a = _lat(dims, L, two_S, 1.0, 0.2, T, 5, eps)
    b = _lat(dims, L, two_S, float(sign), 0.2, T, 5, None)
    sa, sb = a.sweep(12), b.sweep(12)
    assert np.array_equal(a.spins, b.spins)
    for k in ("bond", "mag", "up"):
        # with all eps = -1 the weighted bond sum is -1 times the plain one
        want = sb[k] * (sign if k == "bond" else 1)
        assert np.array_equal(sa[k], want), k


def _enumerate_ea_4x4(eps, J, h, T):
    L, N = 4, 16
    states = np.arange(1 << N, dtype=np.int64)
    s = (((states[:, None] >> np.arange(N)) & 1) * 2 - 1).astype(np.int64)
    e = eps.reshape(2, N).astype(np.int64)
    idx = np.arange(N)
    x, y = idx % L, idx // L
    right = ((x + 1) % L) + L * y
    down = x + L * ((y + 1) % L)
    bond = (e[0] * s * s[:, right]).sum(1) + (e[1] * s * s[:, down]).sum(1)
    mag = s.sum(1)
    E = -J * bond - h * mag
    w = np.exp(-(E - E.min()) / T)
    Z = w.sum()
    return (w * E).sum() / Z / N, (w * np.abs(mag)).sum() / Z / N


@pytest.mark.parametrize("T,h", [(1.5, 0.0), (2.2, 0.4)])
def test_enumeration_random_instance(T, h):
    rng = np.random.default_rng(3)
    eps = rng.choice(np.array([-1, 1], dtype=np.int8), 32)
    E, M = _enumerate_ea_4x4(eps, 1.0, h, T)
    o = _lat(2, 4, 1, 1.0, h, T, 9, eps)
    o.sweep(1000)
    ser = o.sweep(150000)
    e, de = _mean_and_error(o.energy(ser["bond"], ser["mag"]) / 16)
    m, dm = _mean_and_error(np.abs(ser["mag"]) / 16)
    assert abs(e - E) < 5 * de + 1e-4, (e, E, de)
    assert abs(m - M) < 5 * dm + 1e-4, (m, M, dm)


def test_measure_matches_a_recount():
    rng = np.random.default_rng(8)
    L, N = 6, 216
    eps = rng.choice(np.array([-1, 1], dtype=np.int8), 3 * N)
    o = _lat(3, L, 1, 1.0, 0.0, 3.0, 4, eps)
    o.sweep(5)
    s = o.spins.astype(np.int64).reshape(L, L, L)   # [z][y][x]
    e = eps.astype(np.int64).reshape(3, L, L, L)
    bond = (e[0] * s * np.roll(s, -1, axis=2)).sum() + (e[1] * s * np.roll(s, -1, axis=1)).sum() + \
        (e[2] * s * np.roll(s, -1, axis=0)).sum()
    assert o.measure()["bond"] == int(bond)


# ---- per-site field signs (Eq. 1's B_i = h * eta_i) -----------------------

@pytest.mark.parametrize("dims,L", [(2, 8), (3, 6)])
def test_gauge_invariance_with_random_fields(dims, L):
    # tau maps eps_ij -> tau_i tau_j eps_ij and eta_i -> tau_i eta_i: every
    # move keeps its energy change, so the chain is tau*s(t) with h != 0 too
    rng = np.random.default_rng(100 + L)
    N = L ** dims
    eps = rng.choice(np.array([-1, 1], dtype=np.int8), dims * N)
    eta = rng.choice(np.array([-1, 1], dtype=np.int8), N)
    tau = rng.choice(np.array([-1, 1], dtype=np.int8), N)
    a = _lat(dims, L, 1, 1.0, 0.7, 1.4, 33, eps)
    a.set_fields(eta)
    b = _lat(dims, L, 1, 1.0, 0.7, 1.4, 33, _gauge(dims, L, eps, tau), spins=a.spins * tau)
    b.set_fields(eta * tau)
    for _ in range(5):
        sa, sb = a.sweep(3), b.sweep(3)
        assert np.array_equal(b.spins, a.spins * tau)
        assert np.array_equal(sa["bond"], sb["bond"])
        assert np.array_equal(sa["field"], sb["field"])


@pytest.mark.parametrize("sign", [1, -1])
def test_uniform_field_signs_reduce_to_the_plain_field(sign):
    a = _lat(2, 8, 1, 1.0, 0.4, 1.7, 6)
    a.set_fields(np.full(64, sign, dtype=np.int8))
    b = _lat(2, 8, 1, 1.0, 0.4 * sign, 1.7, 6)
    sa, sb = a.sweep(10), b.sweep(10)
    assert np.array_equal(a.spins, b.spins)
    assert np.array_equal(sa["field"], sign * sb["mag"])


def test_enumeration_random_bonds_and_fields():
    rng = np.random.default_rng(12)
    eps = rng.choice(np.array([-1, 1], dtype=np.int8), 32)
    eta = rng.choice(np.array([-1, 1], dtype=np.int8), 16)
    J, h, T = 1.0, 0.6, 1.6
    L, N = 4, 16
    states = np.arange(1 << N, dtype=np.int64)
    s = (((states[:, None] >> np.arange(N)) & 1) * 2 - 1).astype(np.int64)
    e = eps.reshape(2, N).astype(np.int64)
    idx = np.arange(N)
    x, y = idx % L, idx // L
    bond = (e[0] * s * s[:, ((x + 1) % L) + L * y]).sum(1) + (e[1] * s * s[:, x + L * ((y + 1) % L)]).sum(1)
    E = -J * bond - h * (s * eta.astype(np.int64)).sum(1)
    w = np.exp(-(E - E.min()) / T)
    E_ex = (w * E).sum() / w.sum() / N
    o = _lat(2, 4, 1, J, h, T, 14, eps)
    o.set_fields(eta)
    o.sweep(1000)
    ser = o.sweep(150000)
    ev, de = _mean_and_error((-J * ser["bond"] - h * ser["field"]) / N)
    assert abs(ev - E_ex) < 5 * de + 1e-4, (ev, E_ex, de)
