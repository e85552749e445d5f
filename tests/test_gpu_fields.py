"""Per-site random fields (Eq. 1, B_i = h * eta_i with eta_i = +-1: the
random-field Ising model) on the GPU, alone and together with per-bond
couplings: lattices, counters and the field sums sum_i eta_i s_i must equal
the oracle's bit for bit on the 2D wide kernel, the generic kernel (solo
and batched) and through observables; the field signs survive changes of the couplings and
the other way round; unsupported combinations are refused."""
import numpy as np
import pytest

import oracle
import paper_1209_0296_gb300 as lt

pytestmark = pytest.mark.gpu


def _signs(n, seed, p_neg=0.5):
    rng = np.random.default_rng(seed)
    return np.where(rng.random(n) < p_neg, -1, 1).astype(np.int8)


def fld_pair(dims, L, two_S, J, h, T, seed, n, bonds=False, kernel=lt.KERNEL_AUTO, chunks=None, p_neg=0.5):
    N = L ** dims
    eta = _signs(N, seed + 2000, p_neg)
    eps = _signs(dims * N, seed + 1000) if bonds else None
    o = oracle.Lattice(dims, L, two_S, oracle.ISING, J, h, T, seed=seed, init=oracle.INIT_RANDOM)
    o.set_couplings(eps)
    o.set_fields(eta)
    g = lt.Lattice(dims, L, two_S, lt.ISING, J, h, T, seed=seed, init=lt.INIT_RANDOM)
    try:
        g.set_kernel(kernel)
        if bonds:
            g.set_couplings(eps)
        g.set_fields(eta)
        # before any sweep: E from the measured field sum
        m0 = o.measure()
        assert g.observables()["E"] == pytest.approx((-J * m0["bond"] - h * m0["field"]) / N, abs=1e-12)
        ser_o = o.sweep(n)
        for c in (chunks or [n]):
            g.sweep(c)
        assert np.array_equal(g.get_spins(), o.spins)
        ser = g.series(0, n)
        for k in ("bond", "mag", "up"):
            assert np.array_equal(ser[k], ser_o[k]), k
        assert np.array_equal(g.field_series(0, n), ser_o["field"])
        m = o.measure()
        obs = g.observables()
        assert obs["E"] == pytest.approx((-J * m["bond"] - h * m["field"]) / N, abs=1e-12)
        assert obs["M"] == pytest.approx(m["mag"] / N, abs=1e-12)
        return g.get_kernel()["kernel"]
    finally:
        g.close()


@pytest.mark.parametrize("L", [32, 64, 96, 130])
@pytest.mark.parametrize("bonds", [False, True])
@pytest.mark.parametrize("kernel", [lt.KERNEL_AUTO, lt.KERNEL_GENERIC])
def test_2d_spin_half(L, bonds, kernel):
    k = fld_pair(2, L, 1, 1.0, 0.8, 1.6, 10 + L, 25, bonds=bonds, kernel=kernel, chunks=[3, 22])
    wide = kernel == lt.KERNEL_AUTO and L % 32 == 0
    assert k == (lt.KERNEL_WIDE if wide else lt.KERNEL_GENERIC)


def test_wide_with_reference_and_graphs():
    # a long run (graph replays) with the autocorrelation recorded as well
    L, N = 128, 128 * 128
    eta = _signs(N, 9)
    o = oracle.Lattice(2, L, 1, oracle.ISING, 1.0, 1.1, 2.0, seed=9, init=oracle.INIT_RANDOM)
    g = lt.Lattice(2, L, 1, lt.ISING, 1.0, 1.1, 2.0, seed=9, init=lt.INIT_RANDOM)
    o.set_fields(eta)
    g.set_fields(eta)
    ref = o.spins.copy()
    g.set_reference()
    ser_o = o.sweep(70)
    g.sweep(70)
    assert g.get_kernel()["kernel"] == lt.KERNEL_WIDE
    assert np.array_equal(g.get_spins(), o.spins)
    assert np.array_equal(g.field_series(0, 70), ser_o["field"])
    assert g.autocorrelation(69, 1)[0][0] == int(np.dot(o.spins.astype(np.int64), ref))
    g.close()


@pytest.mark.parametrize("dims,L,two_S", [(2, 50, 1), (3, 16, 1), (3, 10, 1), (2, 32, 2), (3, 8, 2), (2, 12, 3),
                                          (3, 6, 7)])
@pytest.mark.parametrize("bonds", [False, True])
def test_generic_sizes_spins_and_3d(dims, L, two_S, bonds):
    fld_pair(dims, L, two_S, 1.0, -0.9, 1.5 * two_S + 0.5, 40 + L + two_S, 20, bonds=bonds)


def test_strong_biased_field():
    # |h| > 4J: each spin mostly follows its own field
    fld_pair(2, 64, 1, 1.0, 5.0, 1.0, 77, 30, p_neg=0.8)


@pytest.mark.slow
def test_full_size_L4096():
    fld_pair(2, 4096, 1, 1.0, 1.0, 1.5, 7, 2, bonds=True)


@pytest.mark.slow
@pytest.mark.parametrize("fields", [False, True])
def test_column_walk_with_reference_L2048(fields):
    # L = 2048: each thread of the one-wave grid walks its chunk column over
    # several rows (some threads one more than others), so the two-chunk
    # pipeline runs its steady state and both exits; couplings always, the
    # field signs when asked, the overlap with the start recorded
    L, N, n = 2048, 2048 * 2048, 3
    eps, eta = _signs(2 * N, 31), _signs(N, 32)
    o = oracle.Lattice(2, L, 1, oracle.ISING, 1.0, 0.7, 1.8, seed=33, init=oracle.INIT_RANDOM)
    g = lt.Lattice(2, L, 1, lt.ISING, 1.0, 0.7, 1.8, seed=33, init=lt.INIT_RANDOM)
    try:
        o.set_couplings(eps)
        g.set_couplings(eps)
        if fields:
            o.set_fields(eta)
            g.set_fields(eta)
        o.set_reference()
        g.set_reference()
        ser_o = o.sweep(n)
        g.sweep(1)
        g.sweep(n - 1)
        assert g.get_kernel()["kernel"] == lt.KERNEL_WIDE
        assert np.array_equal(g.get_spins(), o.spins)
        ser = g.series(0, n)
        for k in ("bond", "mag", "up"):
            assert np.array_equal(ser[k], ser_o[k]), k
        assert np.array_equal(g.autocorrelation(0, n)[0], ser_o["overlap"])
        if fields:
            assert np.array_equal(g.field_series(0, n), ser_o["field"])
    finally:
        g.close()


def test_batch_with_field_lattices():
    cfgs = [(2, 128, 1, 1.0, 0.7, 1.5, 81, False), (2, 96, 1, 1.0, 0.4, 2.0, 82, True),
            (3, 16, 1, 1.0, 1.2, 2.0, 83, False), (2, 50, 1, 1.0, 0.5, 2.2, 84, True),
            (3, 6, 7, 1.0, 1.0, 6.0, 85, False)]   # the largest doubled table: 3D spin-7/2
    lats, ors = [], []
    for dims, L, two_S, J, h, T, seed, bonds in cfgs:
        N = L ** dims
        eta = _signs(N, seed)
        g = lt.Lattice(dims, L, two_S, lt.ISING, J, h, T, seed=seed, init=lt.INIT_RANDOM)
        o = oracle.Lattice(dims, L, two_S, oracle.ISING, J, h, T, seed=seed, init=oracle.INIT_RANDOM)
        if bonds:
            eps = _signs(dims * N, seed + 1)
            g.set_couplings(eps)
            o.set_couplings(eps)
        g.set_fields(eta)
        o.set_fields(eta)
        lats.append(g)
        ors.append(o)
    plain = lt.Lattice(2, 64, 1, lt.ISING, 1.0, 0.0, 2.3, seed=86, init=lt.INIT_RANDOM)
    b = lt.Batch()
    for i, g in enumerate(lats):
        b.add(g, 20 + 3 * i)
    b.add(plain, 17)
    b.run()
    b.synchronize()
    for i, (g, o) in enumerate(zip(lats, ors)):
        n = 20 + 3 * i
        ser_o = o.sweep(n)
        assert np.array_equal(g.get_spins(), o.spins), cfgs[i]
        assert np.array_equal(g.series(0, n)["bond"], ser_o["bond"]), cfgs[i]
        assert np.array_equal(g.field_series(0, n), ser_o["field"]), cfgs[i]
    op = oracle.Lattice(2, 64, 1, oracle.ISING, 1.0, 0.0, 2.3, seed=86, init=oracle.INIT_RANDOM)
    op.sweep(17)
    assert np.array_equal(plain.get_spins(), op.spins)
    b.close()


def test_fields_and_couplings_are_independent():
    L, N = 64, 64 * 64
    eta, eps = _signs(N, 5), _signs(2 * N, 6)
    o = oracle.Lattice(2, L, 1, oracle.ISING, 1.0, 0.6, 2.0, seed=5, init=oracle.INIT_RANDOM)
    g = lt.Lattice(2, L, 1, lt.ISING, 1.0, 0.6, 2.0, seed=5, init=lt.INIT_RANDOM)

    def step(n, first):
        ser_o = o.sweep(n)
        g.sweep(n)
        assert np.array_equal(g.get_spins(), o.spins)
        assert np.array_equal(g.series(first, n)["bond"], ser_o["bond"])
        return ser_o

    o.set_fields(eta)
    g.set_fields(eta)
    step(4, 0)
    o.set_couplings(eps)          # the field signs stay
    g.set_couplings(eps)
    ser_o = step(5, 4)
    assert np.array_equal(g.field_series(4, 5), ser_o["field"])
    o.set_couplings(None)         # still the field signs
    g.set_couplings(None)
    ser_o = step(3, 9)
    assert np.array_equal(g.field_series(0, 12)[9:], ser_o["field"])
    o.set_fields(None)            # uniform again: the wide kernel may take over
    g.set_fields(None)
    g.set_couplings(eps)
    o.set_couplings(eps)
    step(6, 12)
    with pytest.raises(lt.LatticeError):
        g.field_series(12, 6)     # no field signs set
    g.close()


def test_field_series_range_starts_at_the_last_change():
    N = 32 * 32
    g = lt.Lattice(2, 32, 1, lt.ISING, 1.0, 0.5, 2.0, seed=3, init=lt.INIT_RANDOM)
    g.sweep(4)
    g.set_fields(_signs(N, 3))
    g.sweep(5)
    assert g.field_series(4, 5).shape == (5,)
    with pytest.raises(lt.LatticeError):
        g.field_series(3, 2)
    g.close()


def test_refusals():
    N = 64 * 64
    eta = _signs(N, 1)
    ne = lt.Lattice(2, 64, 1, lt.NE, 0.0, 0.0, 0.3, seed=1, init=lt.INIT_EQUILIBRIUM)
    with pytest.raises(lt.LatticeError):
        ne.set_fields(eta)
    ne.close()
    po = lt.Lattice(2, 64, 2, lt.POTTS, 1.0, 0.0, 1.0, seed=1, init=lt.INIT_RANDOM)
    with pytest.raises(lt.LatticeError):
        po.set_fields(eta)
    po.close()
    w3 = lt.Lattice(3, 16, 1, lt.ISING, 1.0, 0.5, 4.0, seed=1, init=lt.INIT_RANDOM)
    w3.set_fields(_signs(16 ** 3, 2))
    with pytest.raises(lt.LatticeError):
        w3.set_kernel(lt.KERNEL_WIDE)   # the 3D wide kernel reads no disorder
    w3.close()
    bp = lt.Lattice(2, 64, 1, lt.ISING, 1.0, 0.0, 2.0, seed=1, init=lt.INIT_RANDOM, layout=lt.BITPACKED)
    with pytest.raises(lt.LatticeError):
        bp.set_fields(eta)
    bp.close()
    g = lt.Lattice(2, 64, 1, lt.ISING, 1.0, 0.5, 2.0, seed=1, init=lt.INIT_RANDOM)
    bad = eta.copy()
    bad[7] = 0
    with pytest.raises(lt.LatticeError):
        g.set_fields(bad)
    g.set_fields(eta)
    for kern in (lt.KERNEL_TILED, lt.KERNEL_RESIDENT):
        with pytest.raises(lt.LatticeError):
            g.set_kernel(kern)
    g.set_kernel(lt.KERNEL_WIDE)
    with pytest.raises(lt.LatticeError):
        g.set_dynamics(lt.DYNAMICS_RANDOM_SITE, 16, 16)
    g.close()
