"""The paper's random-sub-lattice, random-site algorithm (§III.B, second
algorithm) on the GPU: lattices, persistence flags, per-sweep counters and
overlaps must equal the oracle's, integer for integer, for sub-lattice
sizes from 8 to the whole lattice and lambda from 1 to 1024 (both the
one-warp and the many-warp collision paths), for the algorithm and for its
balance-preserving variant."""
import numpy as np
import pytest

import oracle
import paper_1209_0296_gb300 as lt

pytestmark = pytest.mark.gpu


def rs_pair(L, model, Tc, tile, lam, nsweeps, seed=5, chunks=None, ref=True, balanced=False):
    J = 1.0 if model == lt.ISING else 0.0
    init = lt.INIT_RANDOM if model == lt.ISING else lt.INIT_EQUILIBRIUM
    o = oracle.Lattice(2, L, 1, model, J, 0.0, Tc, seed=seed, init=init)
    g = lt.Lattice(2, L, 1, model, J, 0.0, Tc, seed=seed, init=init)
    try:
        g.set_dynamics(lt.DYNAMICS_RANDOM_SITE_BALANCED if balanced else lt.DYNAMICS_RANDOM_SITE, tile, lam)
        if ref:
            g.set_reference()
            o.set_reference()
        ser_o = o.rsite_sweep(nsweeps, tile, lam, balanced=balanced)
        for c in (chunks or [nsweeps]):
            g.sweep(c)
        spins, flags, n = g.get_state()
        assert n == nsweeps
        bad = np.flatnonzero(spins != o.spins)
        assert bad.size == 0, "spins differ at %d sites, first %s" % (bad.size, bad[:8])
        if model == lt.NE:
            assert np.array_equal(flags, o.flags)
        ser = g.series(0, nsweeps)
        for k in ("bond", "mag", "up") + (("unflipped",) if model == lt.NE else ()):
            assert np.array_equal(ser[k], ser_o[k]), k
        if ref:
            ov, _ = g.autocorrelation(0, nsweeps, m=0.0)
            assert np.array_equal(ov, ser_o["overlap"])
    finally:
        g.close()


@pytest.mark.parametrize("L,tile,lam", [(64, 32, 16), (64, 8, 32), (64, 8, 1), (64, 16, 4),
                                        (128, 16, 64), (64, 32, 512), (32, 32, 4), (256, 128, 1024),
                                        (24, 8, 4), (8, 8, 2), (40, 8, 16)])
@pytest.mark.parametrize("model,Tc", [(lt.NE, 0.42), (lt.ISING, 2.3)])
def test_random_site_matches_oracle(L, tile, lam, model, Tc):
    rs_pair(L, model, Tc, tile, lam, 6, seed=L + tile + lam, chunks=[1, 5])


@pytest.mark.parametrize("L,tile,lam", [(64, 32, 16), (64, 8, 8), (64, 8, 1), (64, 16, 4),
                                        (128, 16, 32), (64, 32, 128), (32, 32, 4), (256, 128, 1024),
                                        (24, 8, 2), (8, 8, 8), (40, 8, 4)])
@pytest.mark.parametrize("model,Tc", [(lt.NE, 0.42), (lt.ISING, 2.3)])
def test_balanced_variant_matches_oracle(L, tile, lam, model, Tc):
    rs_pair(L, model, Tc, tile, lam, 5, seed=L + tile + lam + 1, chunks=[2, 3], balanced=True)


def test_balanced_variant_graphs_and_rejections():
    rs_pair(64, lt.ISING, 2.5, 16, 8, 70, chunks=[70], balanced=True, ref=False)   # a graph + direct sweeps
    g = lt.Lattice(2, 64, 1, lt.NE, 0.0, 0.0, 0.3, seed=1, init=lt.INIT_EQUILIBRIUM)
    for tile, lam in ((16, 64), (8, 16), (32, 256)):   # q/2 odd or q < 2
        with pytest.raises(lt.LatticeError):
            g.set_dynamics(lt.DYNAMICS_RANDOM_SITE_BALANCED, tile, lam)
    g.set_dynamics(lt.DYNAMICS_RANDOM_SITE_BALANCED, 16, 32)
    g.close()


def test_serial_limit_whole_lattice():
    # one sub-lattice, one pick per round: serial random-site Metropolis
    rs_pair(64, lt.NE, 0.3, 64, 1, 3)
    rs_pair(32, lt.ISING, 2.0, 32, 1, 3)


def test_whole_lattice_256_with_graphs():
    rs_pair(256, lt.NE, 0.2, 256, 8, 2, ref=False)
    rs_pair(64, lt.ISING, 2.5, 16, 8, 100, chunks=[100])   # a 64-sweep graph + direct sweeps


def test_mixed_dynamics_chain():
    # checkerboard, then random-site, then checkerboard again: one chain
    o = oracle.Lattice(2, 64, 1, lt.NE, 0.0, 0.0, 0.35, seed=9, init=lt.INIT_EQUILIBRIUM)
    g = lt.Lattice(2, 64, 1, lt.NE, 0.0, 0.0, 0.35, seed=9, init=lt.INIT_EQUILIBRIUM)
    o.sweep(7)
    g.sweep(7)
    g.set_dynamics(lt.DYNAMICS_RANDOM_SITE, 16, 16)
    o.rsite_sweep(5, 16, 16)
    g.sweep(5)
    g.set_dynamics(lt.DYNAMICS_CHECKERBOARD)
    ser_o = o.sweep(9)
    g.sweep(9)
    spins, flags, n = g.get_state()
    assert n == 21
    assert np.array_equal(spins, o.spins)
    assert np.array_equal(flags, o.flags)
    assert np.array_equal(g.series(12, 9)["unflipped"], ser_o["unflipped"])
    g.close()


def test_rejections():
    g3 = lt.Lattice(3, 16, 1, lt.ISING, 1.0, 0.0, 4.0, seed=1, init=lt.INIT_RANDOM)
    with pytest.raises(lt.LatticeError):
        g3.set_dynamics(lt.DYNAMICS_RANDOM_SITE, 8, 4)
    g3.close()
    g = lt.Lattice(2, 96, 1, lt.NE, 0.0, 0.0, 0.3, seed=1, init=lt.INIT_EQUILIBRIUM)
    for tile, lam in ((64, 16), (32, 3), (32, 1024), (4, 2), (16, 2048)):
        with pytest.raises(lt.LatticeError):
            g.set_dynamics(lt.DYNAMICS_RANDOM_SITE, tile, lam)
    g.set_dynamics(lt.DYNAMICS_RANDOM_SITE, 32, 16)
    b = lt.Batch()
    with pytest.raises(lt.LatticeError):
        b.add(g, 3)
    b.close()
    g.close()


@pytest.mark.slow
def test_full_size_north_east_L8192():
    # North-East L = 8192, c = 0.42 (the paper's Fig. 5 value), 32x32
    # sub-lattices, lambda = 16, equilibrium start (seed 21): one sweep
    rs_pair(8192, lt.NE, 0.42, 32, 16, 1, seed=21)
