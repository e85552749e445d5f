"""Exact (enumerated) quantities for tiny periodic lattices, written from the
paper's definitions without reference to the oracle's code.

* Boltzmann averages by brute-force enumeration of every configuration
  (canonical weights exp(-H/T), H of Eq. 2 with a field h).
* The exact per-site distribution after one checkerboard sweep: colour-0
  sites move first, each by the single-site Metropolis rule min[1, exp(-dH/T)]
  (§III.A), then colour-1 sites given the new colour-0 values; the North-East
  model (§III.B) only lets a site move when its north and east neighbours are
  up.  These are the paper's rules, evaluated in floating point from the
  rule itself, used to test the oracle's sampled sweeps statistically.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def spin_values(two_S: int) -> np.ndarray:
    if two_S % 2 == 1:
        return np.arange(-two_S, two_S + 1, 2, dtype=np.int64)
    return np.arange(-(two_S // 2), two_S // 2 + 1, dtype=np.int64)


def coords(dims, L):
    """(x, y, z) of linear site i = x + L*(y + L*z)."""
    N = L ** dims
    i = np.arange(N)
    x = i % L
    y = (i // L) % L
    z = i // (L * L) if dims == 3 else np.zeros_like(i)
    return x, y, z


def index(dims, L, x, y, z):
    x, y, z = x % L, y % L, z % L
    return x + L * (y + L * (z if dims == 3 else 0))


def bonds_forward(dims, L):
    """Bond list (i, i+e_d) for every site and direction (each pair per direction once)."""
    x, y, z = coords(dims, L)
    i = np.arange(L ** dims)
    out = [(i, index(dims, L, x + 1, y, z)), (i, index(dims, L, x, y + 1, z))]
    if dims == 3:
        out.append((i, index(dims, L, x, y, z + 1)))
    return out


def neighbours(dims, L):
    x, y, z = coords(dims, L)
    nb = [index(dims, L, x - 1, y, z), index(dims, L, x + 1, y, z),
          index(dims, L, x, y - 1, z), index(dims, L, x, y + 1, z)]
    if dims == 3:
        nb += [index(dims, L, x, y, z - 1), index(dims, L, x, y, z + 1)]
    return np.stack(nb, axis=1)


def enumerate_averages(dims, L, two_S, J, h, T, chunk=1 << 21):
    """Exact <E>/N, <|M|>/N, <M^2>/N^2 over all (2S+1)^N configurations."""
    if dims == 2:
        return _enumerate_rows_2d(L, two_S, J, h, T)
    return enumerate_sites(dims, L, two_S, J, h, T, chunk)


def enumerate_sites(dims, L, two_S, J, h, T, chunk=1 << 21):
    """Site-by-site enumeration (any dims); also checks the 2D row version."""
    vals = spin_values(two_S)
    q = len(vals)
    N = L ** dims
    total = q ** N
    bl = bonds_forward(dims, L)
    Z = 0.0
    sE = sM = sM2 = 0.0
    for start in range(0, total, chunk):
        idx = np.arange(start, min(total, start + chunk), dtype=np.int64)
        digits = np.empty((idx.size, N), dtype=np.int64)
        rem = idx.copy()
        for site in range(N):
            digits[:, site] = rem % q
            rem //= q
        s = vals[digits]
        bond = np.zeros(idx.size, dtype=np.int64)
        for a, b in bl:
            bond += (s[:, a] * s[:, b]).sum(axis=1)
        mag = s.sum(axis=1)
        E = -J * bond - h * mag
        w = np.exp(-E / T)
        Z += w.sum()
        sE += (w * E).sum()
        sM += (w * np.abs(mag)).sum()
        sM2 += (w * mag.astype(np.float64) ** 2).sum()
    return sE / Z / N, sM / Z / N, sM2 / Z / N / N


def _enumerate_rows_2d(L, two_S, J, h, T):
    """Same sums for a 2D L x L lattice, every configuration visited as a
    tuple of L row states (q^L each): H = sum of in-row bonds + bonds between
    consecutive rows (periodic) - h * M."""
    vals = spin_values(two_S)
    q = len(vals)
    R = q ** L
    idx = np.arange(R)
    rows = np.stack([vals[(idx // q ** x) % q] for x in range(L)], axis=1)   # (R, L)
    intra = (rows * np.roll(rows, -1, axis=1)).sum(axis=1)                   # x bonds
    mrow = rows.sum(axis=1)
    inter = rows @ rows.T                                                     # y bonds
    N = L * L
    Z = sE = sM = sM2 = 0.0
    # Sum over the first row explicitly and over the remaining L-1 rows as
    # a full outer product (L = 4: 81 x 81^3 terms for spin-1).
    for r0 in range(R):
        shape = (R,) * (L - 1)
        bond = np.full(shape, intra[r0] + 0, dtype=np.int64)
        mag = np.full(shape, mrow[r0] + 0, dtype=np.int64)
        prev = None
        for k in range(L - 1):
            ax = [1] * (L - 1)
            ax[k] = R
            bond = bond + intra.reshape(ax)
            mag = mag + mrow.reshape(ax)
            if k == 0:
                bond = bond + inter[r0].reshape(ax)
            else:
                ax2 = [1] * (L - 1)
                ax2[k - 1] = R
                ax2[k] = R
                bond = bond + inter.reshape(ax2)
            prev = k
        axl = [1] * (L - 1)
        axl[prev] = R
        bond = bond + inter[:, r0].reshape(axl)
        E = -J * bond - h * mag
        w = np.exp(-E / T)
        Z += w.sum()
        sE += (w * E).sum()
        sM += (w * np.abs(mag)).sum()
        sM2 += (w * mag.astype(np.float64) ** 2).sum()
    return sE / Z / N, sM / Z / N, sM2 / Z / N / N


def _site_dist(k, n, allowed, two_S, J, h, T, cmode, c):
    vals = spin_values(two_S)
    q = len(vals)
    dist = np.zeros(q)
    if not allowed:
        dist[k] = 1.0
        return dist
    props = [1 - k] if two_S == 1 else [k2 for k2 in range(q) if k2 != k]
    w = 1.0 if two_S == 1 else 1.0 / two_S
    stay = 1.0
    for k2 in props:
        ds = vals[k2] - vals[k]
        if cmode:
            p = c / (1 - c) if vals[k2] > vals[k] else (1 - c) / c
        else:
            dE = -J * ds * n - h * ds
            p = math.exp(-dE / T)
        a = min(1.0, p) * w
        dist[k2] += a
        stay -= a
    dist[k] += stay
    return dist


def one_sweep_marginals(dims, L, two_S, model, J, h, T_or_c, state):
    """P[i, k]: exact probability that site i holds state k after one sweep
    from the configuration given as state indices `state` (k per site)."""
    vals = spin_values(two_S)
    q = len(vals)
    N = L ** dims
    cmode = (model == 1 and J == 0.0 and h == 0.0)
    T = None if cmode else T_or_c
    c = T_or_c if cmode else None
    x, y, z = coords(dims, L)
    colour = (x + y + z) & 1
    nb = neighbours(dims, L)
    north = index(dims, L, x, y - 1, z)
    east = index(dims, L, x + 1, y, z)
    c0 = np.flatnonzero(colour == 0)
    c1 = np.flatnonzero(colour == 1)

    def dist_at(i, cfg):
        n = int(vals[cfg[nb[i]]].sum())
        allowed = True
        if model == 1:
            allowed = vals[cfg[north[i]]] == 1 and vals[cfg[east[i]]] == 1
        return _site_dist(int(cfg[i]), n, allowed, two_S, J, h, T, cmode, c)

    state = np.asarray(state, dtype=np.int64)
    d0 = [dist_at(i, state) for i in c0]
    P = np.zeros((N, q))
    for i, d in zip(c0, d0):
        P[i] = d
    supports = [np.flatnonzero(d > 0) for d in d0]
    for combo in itertools.product(*supports):
        w = 1.0
        for d, k in zip(d0, combo):
            w *= d[k]
        if w == 0.0:
            continue
        cfg = state.copy()
        cfg[c0] = combo
        for i in c1:
            P[i] += w * dist_at(i, cfg)
    return P
