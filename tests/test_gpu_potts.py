"""q-state Potts model on the GPU (the 8-sites-per-thread Potts kernel and
the generic kernel, solo and batched): labels, counters and overlaps with a
reference state must equal the oracle's bit for bit; unsupported paths are
refused."""
import numpy as np
import pytest

import oracle
import paper_1209_0296_gb300 as lt

pytestmark = pytest.mark.gpu


def potts_pair(dims, L, q, J, h, T, seed, n, init=lt.INIT_RANDOM, chunks=None, kernel=lt.KERNEL_AUTO,
               ref=False):
    o = oracle.Lattice(dims, L, q - 1, oracle.POTTS, J, h, T, seed=seed, init=init)
    g = lt.Lattice(dims, L, q - 1, lt.POTTS, J, h, T, seed=seed, init=init)
    try:
        g.set_kernel(kernel)
        assert np.array_equal(g.get_spins(), o.spins), "initial labels differ"
        if ref:
            o.set_reference()
            g.set_reference()
        ser_o = o.sweep(n)
        for c in (chunks or [n]):
            g.sweep(c)
        assert np.array_equal(g.get_spins(), o.spins)
        ser = g.series(0, n)
        for k in ("bond", "mag", "up"):
            assert np.array_equal(ser[k], ser_o[k]), k
        m = o.measure()
        obs = g.observables()
        N = L ** dims
        assert obs["E"] == pytest.approx((-J * m["bond"] - h * m["mag"]) / N, abs=1e-12)
        assert obs["M"] == pytest.approx(m["mag"] / N, abs=1e-15)
        if ref:
            assert np.array_equal(g.autocorrelation(0, n)[0], ser_o["overlap"])
        return g.get_kernel()["kernel"]
    finally:
        g.close()


@pytest.mark.parametrize("q", [2, 3, 4, 9])
@pytest.mark.parametrize("dims,L", [(2, 16), (2, 64), (2, 30), (3, 8), (3, 16), (2, 48)])
@pytest.mark.parametrize("kernel", [lt.KERNEL_AUTO, lt.KERNEL_GENERIC])
def test_potts_matches_oracle(q, dims, L, kernel):
    k = potts_pair(dims, L, q, 1.0, 0.2, 0.9 if dims == 2 else 1.6, 3 * q + L, 15, chunks=[2, 13], kernel=kernel)
    fast = kernel == lt.KERNEL_AUTO and L % 16 == 0
    assert k == (lt.KERNEL_WIDE if fast else lt.KERNEL_GENERIC)


@pytest.mark.parametrize("q,dims,L", [(2, 2, 32), (3, 2, 48), (5, 3, 16), (3, 2, 30)])
@pytest.mark.parametrize("kernel", [lt.KERNEL_AUTO, lt.KERNEL_GENERIC])
def test_potts_overlap_series(q, dims, L, kernel):
    potts_pair(dims, L, q, 1.0, 0.0, 1.2, 7 + q, 40, kernel=kernel, ref=True, chunks=[1, 39])


def test_potts_long_run_graphs():
    # graph replays (64 sweeps each at this size) and a direct tail
    potts_pair(2, 64, 4, 1.0, -0.1, 0.8, 41, 150, chunks=[150])


@pytest.mark.slow
def test_potts_full_size_L4096_q3():
    import math
    potts_pair(2, 4096, 3, 1.0, 0.0, 1 / math.log(1 + math.sqrt(3)), 7, 2)


@pytest.mark.slow
@pytest.mark.parametrize("dims,L,q,ref", [(2, 2560, 2, False), (2, 2560, 4, True), (3, 160, 2, True),
                                          (3, 160, 3, False)])
def test_potts_column_walk_several_rows_per_thread(dims, L, q, ref):
    # at these sizes the one-wave grid walks each chunk column over several
    # plane rows (some threads one more than others), so the two-chunk
    # pipeline runs its steady state and both of its exits
    potts_pair(dims, L, q, 1.0, 0.1, 0.9 if dims == 2 else 1.6, 17 + q, 3, chunks=[1, 2], ref=ref)


@pytest.mark.parametrize("init", [lt.INIT_COLD, lt.INIT_RANDOM])
def test_potts_critical_q3(init):
    import math
    potts_pair(2, 128, 3, 1.0, 0.0, 1 / math.log(1 + math.sqrt(3)), 5, 40, init=init)


def test_potts_batch_with_ising():
    cfg_p = [(2, 64, 3, 1.0, 0.0, 1.0, 21, 30), (3, 16, 4, 1.0, 0.1, 1.5, 22, 17), (2, 32, 2, 1.0, 0.0, 1.1, 23, 25)]
    lats, ors = [], []
    for dims, L, q, J, h, T, seed, n in cfg_p:
        lats.append(lt.Lattice(dims, L, q - 1, lt.POTTS, J, h, T, seed=seed, init=lt.INIT_RANDOM))
        ors.append(oracle.Lattice(dims, L, q - 1, oracle.POTTS, J, h, T, seed=seed, init=oracle.INIT_RANDOM))
    ising = lt.Lattice(2, 128, 1, lt.ISING, 1.0, 0.0, 2.3, seed=24, init=lt.INIT_RANDOM)
    b = lt.Batch()
    for g, c in zip(lats, cfg_p):
        b.add(g, c[-1])
    b.add(ising, 20)
    b.run()
    b.synchronize()
    for g, o, c in zip(lats, ors, cfg_p):
        ser_o = o.sweep(c[-1])
        assert np.array_equal(g.get_spins(), o.spins), c
        assert np.array_equal(g.series(0, c[-1])["bond"], ser_o["bond"]), c
    oi = oracle.Lattice(2, 128, 1, oracle.ISING, 1.0, 0.0, 2.3, seed=24, init=oracle.INIT_RANDOM)
    oi.sweep(20)
    assert np.array_equal(ising.get_spins(), oi.spins)
    b.close()


def test_potts_batch_mixed_paths_and_overlaps():
    # Potts items (L % 16 == 0), generic chunks (L = 30, and an explicit
    # generic choice), a reference state on two of them, uneven sweep counts
    cfg = [(2, 48, 3, 0.9, 31, 23, lt.KERNEL_AUTO, True), (2, 30, 4, 0.8, 32, 19, lt.KERNEL_AUTO, False),
           (3, 16, 3, 1.4, 33, 27, lt.KERNEL_AUTO, True), (2, 64, 5, 0.7, 34, 21, lt.KERNEL_GENERIC, False),
           (2, 16, 2, 1.0, 35, 40, lt.KERNEL_AUTO, False)]
    lats, ors = [], []
    for dims, L, q, T, seed, n, kern, ref in cfg:
        g = lt.Lattice(dims, L, q - 1, lt.POTTS, 1.0, 0.1, T, seed=seed, init=lt.INIT_RANDOM)
        o = oracle.Lattice(dims, L, q - 1, oracle.POTTS, 1.0, 0.1, T, seed=seed, init=oracle.INIT_RANDOM)
        g.set_kernel(kern)
        if ref:
            g.set_reference()
            o.set_reference()
        lats.append(g)
        ors.append(o)
    b = lt.Batch()
    for g, c in zip(lats, cfg):
        b.add(g, c[5])
    b.run()
    b.synchronize()
    for g, o, c in zip(lats, ors, cfg):
        n = c[5]
        ser_o = o.sweep(n)
        assert np.array_equal(g.get_spins(), o.spins), c
        ser = g.series(0, n)
        for k in ("bond", "mag", "up"):
            assert np.array_equal(ser[k], ser_o[k]), (c, k)
        if c[7]:
            assert np.array_equal(g.autocorrelation(0, n)[0], ser_o["overlap"]), c
    b.close()
    for g in lats:
        g.close()


@pytest.mark.slow
def test_potts_batch_bands_of_several_rows():
    # eight 2D L = 2048 lattices (and a 3D one) in one batch: enough Potts
    # work that items span several rows per thread (more than one band per
    # lattice, a partial last one on the 3D lattice), q = 2..5, references
    # on some, uneven sweep counts
    cfg = [(2, 2048, 2 + i % 4, 0.8 + 0.05 * i, 50 + i, 1 + i % 2, i % 3 == 0) for i in range(8)]
    cfg.append((3, 48, 3, 1.3, 60, 3, True))
    lats, ors = [], []
    for dims, L, q, T, seed, n, ref in cfg:
        g = lt.Lattice(dims, L, q - 1, lt.POTTS, 1.0, 0.05, T, seed=seed, init=lt.INIT_RANDOM)
        o = oracle.Lattice(dims, L, q - 1, oracle.POTTS, 1.0, 0.05, T, seed=seed, init=oracle.INIT_RANDOM)
        if ref:
            g.set_reference()
            o.set_reference()
        lats.append(g)
        ors.append(o)
    b = lt.Batch()
    for g, c in zip(lats, cfg):
        b.add(g, c[5])
    b.run()
    b.synchronize()
    for g, o, c in zip(lats, ors, cfg):
        n = c[5]
        ser_o = o.sweep(n)
        assert np.array_equal(g.get_spins(), o.spins), c
        ser = g.series(0, n)
        for k in ("bond", "mag", "up"):
            assert np.array_equal(ser[k], ser_o[k]), (c, k)
        if c[6]:
            assert np.array_equal(g.autocorrelation(0, n)[0], ser_o["overlap"]), c
    b.close()
    for g in lats:
        g.close()


def test_potts_labels_and_refusals():
    g = lt.Lattice(2, 16, 2, lt.POTTS, 1.0, 0.0, 1.0, seed=1, init=lt.INIT_RANDOM)
    labels = np.random.default_rng(0).integers(0, 3, 256).astype(np.int8)
    g.set_spins(labels)
    assert np.array_equal(g.get_spins(), labels)
    for bad in (3, -1):
        x = labels.copy()
        x[9] = bad
        with pytest.raises(lt.LatticeError):
            g.set_spins(x)
    assert np.array_equal(g.get_spins(), labels)
    for kern in (lt.KERNEL_TILED, lt.KERNEL_RESIDENT):
        with pytest.raises(lt.LatticeError):
            g.set_kernel(kern)
    g.set_kernel(lt.KERNEL_WIDE)
    g.close()
    odd = lt.Lattice(2, 30, 2, lt.POTTS, 1.0, 0.0, 1.0, seed=1, init=lt.INIT_RANDOM)
    with pytest.raises(lt.LatticeError):
        odd.set_kernel(lt.KERNEL_WIDE)   # L % 16 != 0: generic only
    odd.close()
    q2 = lt.Lattice(2, 64, 1, lt.POTTS, 1.0, 0.0, 1.0, seed=1, init=lt.INIT_RANDOM)
    with pytest.raises(lt.LatticeError):
        q2.set_dynamics(lt.DYNAMICS_RANDOM_SITE, 16, 16)
    with pytest.raises(lt.LatticeError):
        q2.set_couplings(np.ones(2 * 4096, dtype=np.int8))
    q2.close()
    with pytest.raises(lt.LatticeError):
        lt.Lattice(2, 64, 1, lt.POTTS, 1.0, 0.0, 1.0, seed=1, layout=lt.BITPACKED)
