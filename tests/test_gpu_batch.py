"""Batched engine: many uneven lattices advanced together must end bit for
bit where each would end alone, and where the oracle ends.

Mixed batches cover the one-launch tiled sweep (2D spin-1/2, L % 32 == 0,
Ising and North-East), the two-launch wide sweep (3D or spin-S Ising,
L % 16 == 0), the two-launch generic sweep (other sizes), lattices dropping
out at different sweep counts, and graph replays.
"""
import numpy as np
import pytest

import oracle
import paper_1209_0296_gb300 as lt

pytestmark = pytest.mark.gpu

MIX = [
    # dims, L, two_S, model, J, h, T_or_c, seed, init, sweeps
    (2, 64, 1, lt.ISING, 1.0, 0.0, 2.269185, 1234, lt.INIT_COLD, 70),
    (2, 96, 1, lt.ISING, 1.0, 0.1, 2.4, 5, lt.INIT_RANDOM, 37),
    (2, 50, 1, lt.ISING, -0.8, 0.3, 1.9, 6, lt.INIT_RANDOM, 10),
    (3, 8, 2, lt.ISING, 1.0, 0.0, 3.0, 11, lt.INIT_RANDOM, 64),
    (3, 6, 3, lt.ISING, 0.7, 0.2, 9.0, 12, lt.INIT_RANDOM, 33),
    (2, 64, 1, lt.NE, 0.0, 0.0, 0.3, 21, lt.INIT_EQUILIBRIUM, 100),
    (2, 20, 1, lt.NE, 0.0, 0.0, 0.45, 22, lt.INIT_EQUILIBRIUM, 45),
    (2, 288, 1, lt.NE, 0.5, -1.0, 1.5, 23, lt.INIT_RANDOM, 9),
    (2, 32, 1, lt.ISING, 1.0, 0.0, 3.5, 24, lt.INIT_RANDOM, 1),
    (3, 16, 2, lt.ISING, 1.0, 0.0, 3.0, 31, lt.INIT_RANDOM, 40),
    (3, 32, 1, lt.ISING, 1.0, 0.05, 4.2, 32, lt.INIT_COLD, 35),
    (2, 48, 3, lt.ISING, 0.9, -0.2, 5.0, 33, lt.INIT_RANDOM, 66),
    (3, 16, 7, lt.ISING, 1.0, 0.0, 30.0, 34, lt.INIT_RANDOM, 12),
    # 3D / spin-S items: byte-parallel (2D spin-1; bands with a partial last
    # one), and per site where the table has never-accept entries
    (2, 64, 2, lt.ISING, 1.0, 0.1, 1.8, 35, lt.INIT_RANDOM, 20),
    (3, 16, 2, lt.ISING, 1.0, 0.0, 0.25, 36, lt.INIT_RANDOM, 15),
    (3, 16, 1, lt.ISING, 1.0, 0.0, 0.2, 37, lt.INIT_RANDOM, 15),
    (3, 48, 2, lt.ISING, 1.0, 0.0, 3.0, 38, lt.INIT_RANDOM, 7),
    (2, 1024, 2, lt.ISING, 1.0, 0.0, 1.7, 39, lt.INIT_RANDOM, 3),
    (3, 96, 1, lt.ISING, 1.0, 0.0, 4.5, 40, lt.INIT_RANDOM, 3),
]


def _make(c):
    dims, L, two_S, model, J, h, Tc, seed, init, _ = c
    return lt.Lattice(dims, L, two_S, model, J, h, Tc, seed=seed, init=init)


def test_mixed_batch_matches_oracle_and_solo():
    lats = [_make(c) for c in MIX]
    b = lt.Batch()
    for g, c in zip(lats, MIX):
        b.add(g, c[-1])
    b.run()
    b.synchronize()
    for g, c in zip(lats, MIX):
        dims, L, two_S, model, J, h, Tc, seed, init, n = c
        o = oracle.Lattice(dims, L, two_S, model, J, h, Tc, seed=seed, init=init)
        ser_o = o.sweep(n)
        spins, flags, done = g.get_state()
        assert done == n
        assert np.array_equal(spins, o.spins), c
        if model == lt.NE:
            assert np.array_equal(flags, o.flags), c
        ser = g.series(0, n)
        for k in ("bond", "mag", "up") + (("unflipped",) if model == lt.NE else ()):
            assert np.array_equal(ser[k], ser_o[k]), (c, k)
        # and the same as a solo run of the same lattice
        solo = _make(c)
        solo.sweep(n)
        assert np.array_equal(solo.get_spins(), spins)
    b.close()


def test_batch_then_solo_continues_the_same_chain():
    c = MIX[0]
    g = _make(c)
    b = lt.Batch()
    b.add(g, 40)
    b.add(g, 5)          # adds up: 45 sweeps
    b.run()
    g.sweep(15)          # continue alone
    ref = _make(c)
    ref.sweep(60)
    assert g.sweeps() == 60
    assert np.array_equal(g.get_spins(), ref.get_spins())
    assert np.array_equal(g.series(0, 60)["bond"], ref.series(0, 60)["bond"])


def test_three_dimensional_spin_one_batch_full_size():
    # 3D spin-1, L = 256, T_k = 2 + k * 2/15 (seed 11): four of the sixteen
    # temperatures batched for one sweep; two checked against the oracle,
    # all against their solo runs.
    Ts = [2.0 + k * 2.0 / 15 for k in (0, 5, 10, 15)]
    lats = [lt.Lattice(3, 256, 2, lt.ISING, 1.0, 0.0, T, seed=11, init=lt.INIT_RANDOM) for T in Ts]
    b = lt.Batch()
    for g in lats:
        b.add(g, 1)
    b.run()
    for i, (g, T) in enumerate(zip(lats, Ts)):
        s = g.get_spins()
        solo = lt.Lattice(3, 256, 2, lt.ISING, 1.0, 0.0, T, seed=11, init=lt.INIT_RANDOM)
        solo.sweep(1)
        assert np.array_equal(s, solo.get_spins())
        if i in (0, 3):
            o = oracle.Lattice(3, 256, 2, oracle.ISING, 1.0, 0.0, T, seed=11, init=oracle.INIT_RANDOM)
            o.sweep(1)
            assert np.array_equal(s, o.spins)


def test_batch_rejects_bitpacked_and_bad_arguments():
    b = lt.Batch()
    with pytest.raises(lt.LatticeError):
        b.add(lt.Lattice(2, 64, 1, lt.ISING, 1.0, 0.0, 2.0, seed=1, layout=lt.BITPACKED), 3)
    with pytest.raises(lt.LatticeError):
        b.add(_make(MIX[0]), -1)
    b.run()  # empty run is a no-op


def test_many_small_lattices_resident():
    # 160 small 2D spin-1/2 lattices (resident CTAs) with uneven sweep counts,
    # next to two lattices on the step loop; every one equals its solo run,
    # a sample equals the oracle.
    rng = np.random.default_rng(5)
    cfgs = []
    for i in range(160):
        L = int(rng.choice([32, 64, 96, 128]))
        if i % 3 == 0:
            cfgs.append((2, L, 1, lt.NE, 0.0, 0.0, float(rng.uniform(0.05, 0.45)), 1000 + i,
                         lt.INIT_EQUILIBRIUM, int(rng.integers(1, 90))))
        else:
            cfgs.append((2, L, 1, lt.ISING, 1.0, float(rng.uniform(-0.2, 0.2)), float(rng.uniform(1.5, 3.5)),
                         1000 + i, lt.INIT_RANDOM, int(rng.integers(1, 90))))
    cfgs.append((2, 512, 1, lt.ISING, 1.0, 0.0, 2.3, 7, lt.INIT_RANDOM, 50))
    cfgs.append((3, 16, 2, lt.ISING, 1.0, 0.0, 3.0, 8, lt.INIT_RANDOM, 70))
    lats = [_make(c) for c in cfgs]
    b = lt.Batch()
    for g, c in zip(lats, cfgs):
        b.add(g, c[-1])
    b.run()
    b.synchronize()
    for i, (g, c) in enumerate(zip(lats, cfgs)):
        n = c[-1]
        spins, flags, done = g.get_state()
        assert done == n
        solo = _make(c)
        solo.set_kernel(lt.KERNEL_WIDE)
        solo.sweep(n)
        s2, f2, _ = solo.get_state()
        assert np.array_equal(spins, s2), c
        assert np.array_equal(flags, f2), c
        for k in ("bond", "mag", "up", "unflipped"):
            assert np.array_equal(g.series(0, n)[k], solo.series(0, n)[k]), (c, k)
        solo.close()
        if i % 37 == 0:
            o = oracle.Lattice(*c[:7], seed=c[7], init=c[8])
            o.sweep(n)
            assert np.array_equal(spins, o.spins), c
    b.close()


def test_explicit_resident_in_batch_and_stream_order():
    # Lattices on their own streams, the batch on another: with no batch
    # synchronise, work on a lattice's stream still sees the batch's result.
    import torch
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    cfgs = [(2, 256, 1, lt.ISING, 1.0, 0.0, 2.269185, 41, lt.INIT_RANDOM, 33),
            (2, 64, 1, lt.NE, 0.0, 0.0, 0.1, 42, lt.INIT_EQUILIBRIUM, 20),
            (2, 1024, 1, lt.ISING, 1.0, 0.0, 2.5, 43, lt.INIT_RANDOM, 12)]
    lats = [lt.Lattice(*c[:7], seed=c[7], init=c[8], stream=sa) for c in cfgs]
    lats[0].set_kernel(lt.KERNEL_RESIDENT)
    b = lt.Batch(stream=sb)
    for g, c in zip(lats, cfgs):
        b.add(g, c[-1])
    b.run()
    for g, c in zip(lats, cfgs):
        g.sweep(3)            # queued on the lattice's stream after the batch
        o = oracle.Lattice(*c[:7], seed=c[7], init=c[8])
        o.sweep(c[-1] + 3)
        assert np.array_equal(g.get_spins(), o.spins), c
    b.close()


def test_batch_tuner_changes_no_bits():
    # A run long enough to tune (its first phase has >= 192 steps): the
    # batch times its candidates (rows per item, steps per graph) on the
    # run's own steps; every lattice must still end bit for bit where its
    # solo run ends, and the tuned values are reported.
    mix = [(2, 1000, 1, lt.NE, 0.0, 0.0, 0.3, 41, lt.INIT_EQUILIBRIUM),
           (2, 1024, 1, lt.ISING, 1.0, 0.0, 2.3, 42, lt.INIT_RANDOM),
           (2, 202, 1, lt.ISING, 1.0, 0.1, 2.0, 43, lt.INIT_RANDOM),
           (3, 32, 2, lt.ISING, 1.0, 0.0, 3.0, 44, lt.INIT_RANDOM),
           (2, 512, 2, lt.POTTS, 1.0, 0.0, 1.0, 45, lt.INIT_RANDOM)]
    n = 300
    lats = [lt.Lattice(*c[:7], seed=c[7], init=c[8]) for c in mix]
    b = lt.Batch()
    for g in lats:
        b.add(g, n)
    b.run()
    b.synchronize()
    tun = b.tuning()
    assert tun["steps_per_graph"] in (8, 32) and tun["rows_per_item"] in (2, 8)
    for g, c in zip(lats, mix):
        solo = lt.Lattice(*c[:7], seed=c[7], init=c[8])
        solo.sweep(n)
        assert g.sweeps() == n
        assert np.array_equal(g.get_spins(), solo.get_spins()), c
        assert np.array_equal(g.series(0, n)["bond"], solo.series(0, n)["bond"]), c
    # a second run of the same composition takes the tuned values without tuning
    for g in lats:
        b.add(g, 20)
    b.run()
    b.synchronize()
    assert b.tuning() == tun
    b.close()
