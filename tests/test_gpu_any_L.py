"""2D spin-1/2 sweeps at any even L (not only multiples of 32).

For L % 32 != 0 the library runs the wide kernel's sweep on single Philox
groups: a plane row of L/2 bytes then need not start on a word boundary
(L % 8 != 0) and its last group holds L/2 % 4 sites.  Every residue of L
modulo 8 and 32, both models (Ising with a field, North-East in c-mode),
with and without a reference state, solo and batched, must match the CPU
oracle bit for bit: spins, persistence flags and every per-sweep counter.
"""
import numpy as np
import pytest

import oracle
import paper_1209_0296_gb300 as lt

pytestmark = pytest.mark.gpu

SIZES = [2, 4, 6, 10, 34, 36, 38, 40, 42, 50, 66, 98, 130, 258, 1000, 1026]


def _pair(L, model, n, kernel=lt.KERNEL_AUTO, ref_at=None, seed=None):
    if model == lt.NE:
        args = (2, L, 1, lt.NE, 0.0, 0.0, 0.3, 21 + L if seed is None else seed, lt.INIT_EQUILIBRIUM)
    else:
        args = (2, L, 1, lt.ISING, 1.0, 0.15, 2.4, 9 + L if seed is None else seed, lt.INIT_RANDOM)
    dims, L_, two_S, mdl, J, h, Tc, sd, init = args
    o = oracle.Lattice(dims, L_, two_S, mdl, J, h, Tc, seed=sd, init=init)
    g = lt.Lattice(dims, L_, two_S, mdl, J, h, Tc, seed=sd, init=init)
    try:
        g.set_kernel(kernel)
        ser_o = {}
        if ref_at is not None:
            o.sweep(ref_at)
            o.set_reference()
            g.sweep(ref_at)
            g.set_reference()
            n_rest = n - ref_at
            ser_o = o.sweep(n_rest)
            g.sweep(n_rest)
            ser = g.series(ref_at, n_rest)
            ov, _ = g.autocorrelation(ref_at, n_rest, m=0.0)
            assert np.array_equal(ov, ser_o["overlap"])
        else:
            ser_o = o.sweep(n)
            g.sweep(n)
            ser = g.series(0, n)
        spins, flags, done = g.get_state()
        assert done == n
        bad = np.flatnonzero(spins != o.spins)
        assert bad.size == 0, "L=%d: spins differ at %d sites, first %s" % (L, bad.size, bad[:8])
        keys = ("bond", "mag", "up")
        if mdl == lt.NE:
            assert np.array_equal(flags, o.flags), "persistence flags differ"
            keys += ("unflipped",)
        for k in keys:
            assert np.array_equal(ser[k], ser_o[k]), (L, k)
        return g.get_kernel()
    finally:
        g.close()


@pytest.mark.parametrize("L", SIZES)
@pytest.mark.parametrize("model", [lt.ISING, lt.NE])
def test_any_L_matches_oracle(L, model):
    n = 20 if L < 500 else 4
    info = _pair(L, model, n)
    assert info["kernel"] == lt.KERNEL_WIDE     # not the generic fallback


@pytest.mark.parametrize("L", [6, 38, 130])
@pytest.mark.parametrize("model", [lt.ISING, lt.NE])
def test_any_L_with_reference_state(L, model):
    _pair(L, model, 14, ref_at=3)


def test_any_L_full_size():
    _pair(4098, lt.ISING, 3)
    _pair(8194, lt.NE, 1)


def test_any_L_batched_matches_oracle():
    rng = np.random.default_rng(5)
    cases = []
    for i, L in enumerate([2, 6, 10, 34, 50, 66, 100, 130, 258, 514, 1030, 64, 96]):
        model = lt.NE if i % 3 == 1 else lt.ISING
        n = int(rng.integers(3, 40))
        cases.append((L, model, n, 300 + i))
    lats, orc = [], []
    b = lt.Batch()
    for L, model, n, seed in cases:
        if model == lt.NE:
            a = (2, L, 1, lt.NE, 0.0, 0.0, 0.25, seed, lt.INIT_EQUILIBRIUM)
        else:
            a = (2, L, 1, lt.ISING, 1.0, -0.1, 2.2, seed, lt.INIT_RANDOM)
        g = lt.Lattice(*a[:7], seed=a[7], init=a[8])
        b.add(g, n)
        lats.append(g)
        orc.append(oracle.Lattice(*a[:7], seed=a[7], init=a[8]))
    b.run()
    b.synchronize()
    for (L, model, n, _), g, o in zip(cases, lats, orc):
        ser_o = o.sweep(n)
        spins, flags, done = g.get_state()
        assert done == n
        assert np.array_equal(spins, o.spins), L
        if model == lt.NE:
            assert np.array_equal(flags, o.flags), L
        ser = g.series(0, n)
        for k in ("bond", "mag", "up") + (("unflipped",) if model == lt.NE else ()):
            assert np.array_equal(ser[k], ser_o[k]), (L, k)
        g.close()
    b.close()
