"""GPU parity: the CUDA library against the CPU oracle, bit for bit.

Every case creates the same lattice on both sides from the same seed, runs
the same number of checkerboard sweeps (§III.A steps 5-8; §III.B rule) and
requires identical int8 spins, identical persistence flags (North-East) and
identical per-sweep int64 counters.  Integer work, so the tolerance is zero.
"""
import numpy as np
import pytest

import oracle
import paper_1209_0296_gb300 as lt

pytestmark = pytest.mark.gpu


def run_pair(dims, L, two_S, model, J, h, Tc, seed, init, nsweeps, kernel=lt.KERNEL_AUTO,
             tile=(0, 0), graph=0, chunks=None):
    o = oracle.Lattice(dims, L, two_S, model, J, h, Tc, seed=seed, init=init)
    g = lt.Lattice(dims, L, two_S, model, J, h, Tc, seed=seed, init=init)
    try:
        assert np.array_equal(g.get_spins(), o.spins), "initial state differs"
        g.set_kernel(kernel, tile[0], tile[1], graph)
        ser_o = o.sweep(nsweeps)
        for c in (chunks or [nsweeps]):
            g.sweep(c)
        ser_g = g.series(0, nsweeps)
        spins, flags, n = g.get_state()
        assert n == nsweeps
        bad = np.flatnonzero(spins != o.spins)
        assert bad.size == 0, "spins differ at %d sites, first %s" % (bad.size, bad[:8])
        if model == lt.NE:
            assert np.array_equal(flags, o.flags), "persistence flags differ"
        keys = ("bond", "mag", "up", "unflipped") if model == lt.NE else ("bond", "mag", "up")
        for k in keys:
            assert np.array_equal(ser_g[k], ser_o[k]), k
        return g, o, ser_g
    finally:
        g.close()


def test_config_L64_cold_1000_sweeps_tiled():
    # 2D Ising spin-1/2, L=64, J=1, h=0, T=2.269185, cold start, seed 1234,
    # 1000 sweeps with per-sweep E and M (every counter compared).
    run_pair(2, 64, 1, lt.ISING, 1.0, 0.0, 2.269185, 1234, lt.INIT_COLD, 1000)


def test_config_L64_cold_1000_sweeps_wide():
    run_pair(2, 64, 1, lt.ISING, 1.0, 0.0, 2.269185, 1234, lt.INIT_COLD, 1000,
             kernel=lt.KERNEL_WIDE)


def test_config_L64_cold_1000_sweeps_generic():
    run_pair(2, 64, 1, lt.ISING, 1.0, 0.0, 2.269185, 1234, lt.INIT_COLD, 1000,
             kernel=lt.KERNEL_GENERIC)


@pytest.mark.parametrize("L", [2, 4, 6, 8, 10, 16, 32, 48])
@pytest.mark.parametrize("T,J,h", [(1.5, 1.0, 0.0), (2.269185, 1.0, 0.2), (3.5, -0.8, -0.3)])
def test_2d_spin_half_small(L, T, J, h):
    for kernel in (lt.KERNEL_GENERIC, lt.KERNEL_AUTO) + ((lt.KERNEL_TILED,) if L % 32 == 0 else ()):
        run_pair(2, L, 1, lt.ISING, J, h, T, 100 + L, lt.INIT_RANDOM, 25, kernel=kernel)


@pytest.mark.parametrize("L,tile", [(288, (256, 32)), (544, (256, 32)), (544, (256, 8)),
                                    (544, (256, 64)), (96, (256, 2)), (4128, (256, 48)),
                                    (64, (256, 7)), (32, (256, 64))])
def test_tiled_ragged_tiles(L, tile):
    n = 12 if L < 4000 else 3
    run_pair(2, L, 1, lt.ISING, 1.0, 0.1, 2.4, 7 + L, lt.INIT_RANDOM, n, kernel=lt.KERNEL_TILED,
             tile=tile)


@pytest.mark.parametrize("L", [32, 64, 96, 288, 4128])
def test_wide_sizes(L):
    n = 12 if L < 4000 else 3
    run_pair(2, L, 1, lt.ISING, 1.0, 0.1, 2.4, 9 + L, lt.INIT_RANDOM, n, kernel=lt.KERNEL_WIDE)
    run_pair(2, L, 1, lt.NE, 0.0, 0.0, 0.35, 9 + L, lt.INIT_EQUILIBRIUM, n, kernel=lt.KERNEL_WIDE)


@pytest.mark.parametrize("two_S", [1, 2, 3, 4, 8])
@pytest.mark.parametrize("L", [2, 4, 6, 10])
def test_3d_spin_S(two_S, L):
    T = 2.0 * max(1, two_S) ** 1.2
    run_pair(3, L, two_S, lt.ISING, 1.0, 0.15, T, 11 + L, lt.INIT_RANDOM, 20)


@pytest.mark.parametrize("two_S", [2, 3, 5])
def test_2d_spin_S(two_S):
    run_pair(2, 12, two_S, lt.ISING, 0.9, -0.1, 1.7 * two_S, 5, lt.INIT_RANDOM, 30)


@pytest.mark.parametrize("dims,L,two_S", [(3, 16, 1), (3, 16, 2), (3, 32, 3), (3, 16, 8),
                                          (2, 16, 2), (2, 48, 4), (2, 64, 7), (3, 48, 2)])
def test_wide_three_d_and_spin_S(dims, L, two_S):
    T = 2.0 * max(1, two_S) ** 1.2
    for kernel in (lt.KERNEL_WIDE, lt.KERNEL_AUTO):
        run_pair(dims, L, two_S, lt.ISING, 1.0, 0.15, T, 13 + L + two_S, lt.INIT_RANDOM, 15,
                 kernel=kernel)


@pytest.mark.parametrize("L", [4, 16, 48, 64, 288])
@pytest.mark.parametrize("c", [0.05, 0.3, 0.45, 0.7])
def test_north_east_c_mode(L, c):
    for kernel in (lt.KERNEL_GENERIC, lt.KERNEL_AUTO) + ((lt.KERNEL_TILED,) if L % 32 == 0 else ()):
        run_pair(2, L, 1, lt.NE, 0.0, 0.0, c, 21 + L, lt.INIT_EQUILIBRIUM, 30, kernel=kernel)


@pytest.mark.parametrize("L", [8, 32, 64])
def test_north_east_temperature_mode(L):
    for kernel in (lt.KERNEL_GENERIC, lt.KERNEL_AUTO) + ((lt.KERNEL_TILED,) if L % 32 == 0 else ()):
        run_pair(2, L, 1, lt.NE, 0.5, -1.0, 1.5, 3, lt.INIT_RANDOM, 30, kernel=kernel)


def test_graph_replay_and_direct_launch_paths_agree():
    # Graph replays (64 sweeps each for this size) and direct launches mixed.
    run_pair(2, 32, 1, lt.ISING, 1.0, 0.0, 2.2, 9, lt.INIT_RANDOM, 333,
             chunks=[1, 63, 64, 200, 5])
    run_pair(3, 8, 2, lt.ISING, 1.0, 0.0, 2.5, 9, lt.INIT_RANDOM, 150, graph=16,
             chunks=[7, 16, 100, 27])


def test_checkpoint_resume_is_bit_exact():
    args = (2, 48, 1, lt.NE, 0.0, 0.0, 0.35, 77, lt.INIT_EQUILIBRIUM)
    a = lt.Lattice(*args[:7], seed=args[7], init=args[8])
    a.sweep(40)
    full = a.get_state()
    b = lt.Lattice(*args[:7], seed=args[7], init=args[8])
    b.sweep(17)
    s, f, n = b.get_state()
    c = lt.Lattice(*args[:7], seed=args[7], init=args[8])
    c.set_state(s, f, n)
    c.sweep(23)
    resumed = c.get_state()
    assert resumed[2] == 40
    assert np.array_equal(resumed[0], full[0]) and np.array_equal(resumed[1], full[1])
    assert np.array_equal(c.series(17, 23)["unflipped"], a.series(17, 23)["unflipped"])
    with pytest.raises(lt.LatticeError):
        c.series(0, 5)   # sweeps before the restore point are not recorded here


def test_observables_follow_series():
    g = lt.Lattice(2, 64, 1, lt.ISING, 1.0, 0.3, 2.1, seed=4, init=lt.INIT_RANDOM)
    o0 = g.observables()
    s = g.get_spins().astype(np.int64).reshape(64, 64)
    bond = int((s * np.roll(s, -1, 1)).sum() + (s * np.roll(s, -1, 0)).sum())
    assert o0["E"] == pytest.approx((-bond - 0.3 * s.sum()) / 4096)
    assert o0["M"] == pytest.approx(s.sum() / 4096)
    g.sweep(10)
    ser = g.series(9, 1)
    o = g.observables()
    assert o["E"] == pytest.approx((-ser["bond"][0] - 0.3 * ser["mag"][0]) / 4096)
    assert o["density"] == pytest.approx(ser["up"][0] / 4096)
    assert np.isnan(o["persistence"])


def test_set_spins_roundtrip_and_validation():
    g = lt.Lattice(3, 6, 2, lt.ISING, 1.0, 0.0, 2.0, seed=1, init=lt.INIT_RANDOM)
    rng = np.random.default_rng(0)
    s = rng.integers(-1, 2, 216).astype(np.int8)
    g.set_spins(s)
    assert np.array_equal(g.get_spins(), s)
    with pytest.raises(lt.LatticeError):
        g.set_spins(np.full(216, 2, dtype=np.int8))
    assert np.array_equal(g.get_spins(), s)          # a rejected array changes nothing
    # one bad byte among good ones; odd parity for half-integer spin; bit-packed
    bad = s.copy()
    bad[100] = -2
    with pytest.raises(lt.LatticeError):
        g.set_spins(bad)
    assert np.array_equal(g.get_spins(), s)
    h = lt.Lattice(2, 8, 3, lt.ISING, 1.0, 0.0, 4.0, seed=1, init=lt.INIT_RANDOM)
    good = rng.choice(np.array([-3, -1, 1, 3], dtype=np.int8), 64)
    h.set_spins(good)
    assert np.array_equal(h.get_spins(), good)
    even = good.copy()
    even[5] = 2
    with pytest.raises(lt.LatticeError):
        h.set_spins(even)
    assert np.array_equal(h.get_spins(), good)
    k = lt.Lattice(2, 64, 1, lt.ISING, 1.0, 0.0, 2.0, seed=1, init=lt.INIT_RANDOM, layout=lt.BITPACKED)
    pm = rng.choice(np.array([-1, 1], dtype=np.int8), 4096)
    k.set_spins(pm)
    assert np.array_equal(k.get_spins(), pm)
    zero = pm.copy()
    zero[7] = 0
    with pytest.raises(lt.LatticeError):
        k.set_spins(zero)
    assert np.array_equal(k.get_spins(), pm)


def test_allocation_failure_is_reported():
    lib = lt.load()
    lib.lattice_test_fail_alloc(2)  # second allocation of the next create fails
    with pytest.raises(lt.LatticeError) as e:
        lt.Lattice(2, 64, 1, lt.ISING, 1.0, 0.0, 2.0, seed=1)
    assert e.value.code == -2
    lib.lattice_test_fail_alloc(0)
    lt.Lattice(2, 64, 1, lt.ISING, 1.0, 0.0, 2.0, seed=1).sweep(3)   # still usable


# ---- full sizes, in the launch configuration the benchmark times ----------

@pytest.mark.parametrize("dims,L,two_S,T,J,h", [(3, 32, 1, 0.2, 1.0, 0.0), (3, 32, 2, 0.25, 1.0, 0.1),
                                                  (2, 64, 2, 0.25, 1.0, 0.0), (3, 16, 2, 0.25, -1.0, 0.0)])
def test_wide_three_d_never_accept_tables(dims, L, two_S, T, J, h):
    # So cold that some moves have p < 2^-32 (thr = 0): the byte-parallel
    # spin-1/2 / spin-1 step, whose t' = thr - 1 table cannot hold such an
    # entry, must give way to the per-site step, still bit-exact
    run_pair(dims, L, two_S, lt.ISING, J, h, T, 29 + L, lt.INIT_RANDOM, 12, kernel=lt.KERNEL_WIDE)


@pytest.mark.slow
@pytest.mark.parametrize("dims,L,two_S,T,J,h,ref", [(3, 160, 1, 4.0, 1.0, 0.2, True),
                                                    (3, 160, 2, 3.0, 1.0, -0.1, False),
                                                    (2, 2048, 2, 1.7, 1.0, 0.1, True),
                                                    (3, 160, 2, 2.0, -1.0, 0.3, True)])
def test_wide_three_d_column_walk_several_rows(dims, L, two_S, T, J, h, ref):
    # sizes at which each thread of the one-wave grid walks its chunk column
    # over several rows (some one more than others): the two-chunk pipeline's
    # steady state and both exits, with and without the overlap counter
    o = oracle.Lattice(dims, L, two_S, lt.ISING, J, h, T, seed=41, init=oracle.INIT_RANDOM)
    g = lt.Lattice(dims, L, two_S, lt.ISING, J, h, T, seed=41, init=lt.INIT_RANDOM)
    try:
        g.set_kernel(lt.KERNEL_WIDE)
        if ref:
            o.set_reference()
            g.set_reference()
        ser_o = o.sweep(3)
        g.sweep(1)
        g.sweep(2)
        assert np.array_equal(g.get_spins(), o.spins)
        ser = g.series(0, 3)
        for k in ("bond", "mag", "up"):
            assert np.array_equal(ser[k], ser_o[k]), k
        if ref:
            assert np.array_equal(g.autocorrelation(0, 3)[0], ser_o["overlap"])
    finally:
        g.close()


@pytest.mark.parametrize("kernel", [lt.KERNEL_TILED, lt.KERNEL_WIDE])
def test_full_size_2d_L4096_random(kernel):
    # 2D Ising spin-1/2, L=4096, T=2.0, random +-1 start (seed 7).
    run_pair(2, 4096, 1, lt.ISING, 1.0, 0.0, 2.0, 7, lt.INIT_RANDOM, 3, kernel=kernel)


@pytest.mark.parametrize("kernel", [lt.KERNEL_GENERIC, lt.KERNEL_WIDE])
def test_full_size_3d_L256_spin_one(kernel):
    # 3D spin-1, L=256, T=2.0 + 7*(2/15), uniform random start (seed 11).
    run_pair(3, 256, 2, lt.ISING, 1.0, 0.0, 2.0 + 7 * 2.0 / 15, 11, lt.INIT_RANDOM, 1, kernel=kernel)


@pytest.mark.parametrize("kernel", [lt.KERNEL_TILED, lt.KERNEL_WIDE])
def test_full_size_north_east_L8192(kernel):
    run_pair(2, 8192, 1, lt.NE, 0.0, 0.0, 0.3, 21, lt.INIT_EQUILIBRIUM, 1, kernel=kernel)


def test_full_size_properties_after_many_sweeps():
    # Beyond what the oracle can follow: every counter must match a direct
    # recount of the final lattice, and spins stay in {-1, +1}.
    L = 4096
    g = lt.Lattice(2, L, 1, lt.ISING, 1.0, 0.0, 2.269185, seed=7, init=lt.INIT_RANDOM)
    g.sweep(300)
    s = g.get_spins()
    assert set(np.unique(s).tolist()) <= {-1, 1}
    s = s.astype(np.int64).reshape(L, L)
    ser = g.series(299, 1)
    assert ser["bond"][0] == (s * np.roll(s, -1, 1)).sum() + (s * np.roll(s, -1, 0)).sum()
    assert ser["mag"][0] == s.sum()
    assert ser["up"][0] == (s > 0).sum()


def test_never_accept_table_falls_back_to_generic():
    # At T = 0.3 a dE = 8 move has p < 2^-32 (thr = 0): the tiled kernel's
    # t' = thr - 1 encoding cannot hold it, so the library must refuse the
    # tiled kernel and the automatic choice must still be bit-exact.
    g = lt.Lattice(2, 64, 1, lt.ISING, 1.0, 0.0, 0.3, seed=3, init=lt.INIT_RANDOM)
    with pytest.raises(lt.LatticeError) as e:
        g.set_kernel(lt.KERNEL_TILED)
    assert e.value.code == -6
    run_pair(2, 64, 1, lt.ISING, 1.0, 0.0, 0.3, 3, lt.INIT_RANDOM, 20)


# ---- resident kernel: the whole lattice in one CTA's shared memory ----------

def test_config_L64_cold_1000_sweeps_resident():
    run_pair(2, 64, 1, lt.ISING, 1.0, 0.0, 2.269185, 1234, lt.INIT_COLD, 1000,
             kernel=lt.KERNEL_RESIDENT)


@pytest.mark.parametrize("L", [32, 64, 96, 128, 224, 448])
def test_resident_ising(L):
    # odd sweep counts per call: the final state alternates between buffers
    run_pair(2, L, 1, lt.ISING, 1.0, 0.1, 2.4, 300 + L, lt.INIT_RANDOM, 45,
             kernel=lt.KERNEL_RESIDENT, chunks=[7, 1, 30, 7])


@pytest.mark.parametrize("L,c", [(32, 0.3), (64, 0.05), (160, 0.2), (416, 0.45)])
def test_resident_north_east(L, c):
    run_pair(2, L, 1, lt.NE, 0.0, 0.0, c, 400 + L, lt.INIT_EQUILIBRIUM, 41,
             kernel=lt.KERNEL_RESIDENT, chunks=[1, 13, 27])


def test_resident_north_east_with_field():
    run_pair(2, 96, 1, lt.NE, 0.5, -1.0, 1.5, 23, lt.INIT_RANDOM, 20, kernel=lt.KERNEL_RESIDENT)


def test_resident_interleaved_with_other_kernels():
    # sweeps alternate between the resident, wide and tiled kernels on one
    # lattice; the chain must be the oracle's
    for model, Tc, init in ((lt.ISING, 2.269185, lt.INIT_RANDOM), (lt.NE, 0.2, lt.INIT_EQUILIBRIUM)):
        J = 1.0 if model == lt.ISING else 0.0
        o = oracle.Lattice(2, 128, 1, model, J, 0.0, Tc, seed=77, init=init)
        g = lt.Lattice(2, 128, 1, model, J, 0.0, Tc, seed=77, init=init)
        ser_o = o.sweep(60)
        for kern, n in ((lt.KERNEL_RESIDENT, 9), (lt.KERNEL_WIDE, 5), (lt.KERNEL_RESIDENT, 20),
                        (lt.KERNEL_TILED, 3), (lt.KERNEL_RESIDENT, 23)):
            g.set_kernel(kern)
            g.sweep(n)
        spins, flags, n = g.get_state()
        assert n == 60
        assert np.array_equal(spins, o.spins)
        if model == lt.NE:
            assert np.array_equal(flags, o.flags)
        ser = g.series(0, 60)
        for k in ("bond", "mag", "up") + (("unflipped",) if model == lt.NE else ()):
            assert np.array_equal(ser[k], ser_o[k]), k
        g.close()


def test_resident_rejects_what_does_not_fit():
    for args in ((2, 480, 1, lt.ISING, 1.0, 0.0, 2.0), (2, 448, 1, lt.NE, 0.0, 0.0, 0.2),
                 (3, 32, 1, lt.ISING, 1.0, 0.0, 4.0), (2, 64, 2, lt.ISING, 1.0, 0.0, 2.0),
                 (2, 80, 1, lt.ISING, 1.0, 0.0, 2.0)):
        g = lt.Lattice(*args, seed=1, init=lt.INIT_RANDOM)
        with pytest.raises(lt.LatticeError):
            g.set_kernel(lt.KERNEL_RESIDENT)
        g.close()
