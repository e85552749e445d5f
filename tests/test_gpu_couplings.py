"""Per-bond couplings (Eq. 1, J_ij = J * eps_ij: the +-J spin glass) on the
GPU: lattices and weighted counters must equal the oracle's bit for bit on
the 2D wide kernel (and its batched form), the generic kernel (3D, spin-S,
other sizes, batched) and through observables; unsupported combinations are
refused."""
import numpy as np
import pytest

import oracle
import paper_1209_0296_gb300 as lt

pytestmark = pytest.mark.gpu


def _eps(dims, L, seed, p_neg=0.5):
    rng = np.random.default_rng(seed)
    return np.where(rng.random(dims * L ** dims) < p_neg, -1, 1).astype(np.int8)


def cpl_pair(dims, L, two_S, J, h, T, seed, n, kernel=lt.KERNEL_AUTO, chunks=None, p_neg=0.5):
    eps = _eps(dims, L, seed + 1000, p_neg)
    o = oracle.Lattice(dims, L, two_S, oracle.ISING, J, h, T, seed=seed, init=oracle.INIT_RANDOM)
    o.set_couplings(eps)
    g = lt.Lattice(dims, L, two_S, lt.ISING, J, h, T, seed=seed, init=lt.INIT_RANDOM)
    try:
        g.set_couplings(eps)
        g.set_kernel(kernel)
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
        return g.get_kernel()["kernel"]
    finally:
        g.close()


@pytest.mark.parametrize("L", [32, 64, 96, 128])
@pytest.mark.parametrize("kernel", [lt.KERNEL_AUTO, lt.KERNEL_GENERIC])
def test_2d_spin_half(L, kernel):
    k = cpl_pair(2, L, 1, 1.0, 0.2, 1.8, 10 + L, 25, kernel=kernel, chunks=[3, 22])
    assert k == (lt.KERNEL_WIDE if kernel == lt.KERNEL_AUTO else lt.KERNEL_GENERIC)


@pytest.mark.parametrize("dims,L,two_S", [(2, 50, 1), (3, 16, 1), (3, 10, 1), (2, 32, 2), (3, 8, 2), (2, 12, 3)])
def test_generic_sizes_spins_and_3d(dims, L, two_S):
    cpl_pair(dims, L, two_S, 1.0, -0.3, 1.5 * two_S + 0.5, 40 + L + two_S, 20)


def test_antiferro_biased_couplings():
    cpl_pair(2, 64, 1, 0.7, 0.0, 1.2, 77, 30, p_neg=0.9)


@pytest.mark.slow
def test_full_size_L4096():
    cpl_pair(2, 4096, 1, 1.0, 0.0, 1.0, 7, 2)


def test_batch_with_coupled_lattices():
    cfgs = [(2, 128, 1, 1.0, 0.0, 1.5, 81), (2, 96, 1, 1.0, 0.1, 2.0, 82), (3, 16, 1, 1.0, 0.0, 2.0, 83),
            (2, 50, 1, 1.0, 0.0, 2.2, 84), (2, 64, 2, 1.0, 0.0, 3.0, 85)]
    lats, ors = [], []
    for dims, L, two_S, J, h, T, seed in cfgs:
        eps = _eps(dims, L, seed)
        g = lt.Lattice(dims, L, two_S, lt.ISING, J, h, T, seed=seed, init=lt.INIT_RANDOM)
        g.set_couplings(eps)
        o = oracle.Lattice(dims, L, two_S, oracle.ISING, J, h, T, seed=seed, init=oracle.INIT_RANDOM)
        o.set_couplings(eps)
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
        ser_o = o.sweep(20 + 3 * i)
        assert np.array_equal(g.get_spins(), o.spins), cfgs[i]
        assert np.array_equal(g.series(0, 20 + 3 * i)["bond"], ser_o["bond"]), cfgs[i]
    op = oracle.Lattice(2, 64, 1, oracle.ISING, 1.0, 0.0, 2.3, seed=86, init=oracle.INIT_RANDOM)
    op.sweep(17)
    assert np.array_equal(plain.get_spins(), op.spins)
    b.close()


def test_clear_couplings_mid_run():
    eps = _eps(2, 64, 5)
    o = oracle.Lattice(2, 64, 1, oracle.ISING, 1.0, 0.0, 2.0, seed=5, init=oracle.INIT_RANDOM)
    g = lt.Lattice(2, 64, 1, lt.ISING, 1.0, 0.0, 2.0, seed=5, init=lt.INIT_RANDOM)
    o.set_couplings(eps)
    g.set_couplings(eps)
    o.sweep(6)
    g.sweep(6)
    o.set_couplings(None)
    g.set_couplings(None)
    ser_o = o.sweep(9)
    g.sweep(9)
    assert np.array_equal(g.get_spins(), o.spins)
    assert np.array_equal(g.series(6, 9)["bond"], ser_o["bond"])
    g.close()


def test_refusals():
    eps2 = _eps(2, 64, 1)
    ne = lt.Lattice(2, 64, 1, lt.NE, 0.0, 0.0, 0.3, seed=1, init=lt.INIT_EQUILIBRIUM)
    with pytest.raises(lt.LatticeError):
        ne.set_couplings(eps2)
    ne.close()
    bp = lt.Lattice(2, 64, 1, lt.ISING, 1.0, 0.0, 2.0, seed=1, init=lt.INIT_RANDOM, layout=lt.BITPACKED)
    with pytest.raises(lt.LatticeError):
        bp.set_couplings(eps2)
    bp.close()
    g = lt.Lattice(2, 64, 1, lt.ISING, 1.0, 0.0, 2.0, seed=1, init=lt.INIT_RANDOM)
    bad = eps2.copy()
    bad[3] = 0
    with pytest.raises(lt.LatticeError):
        g.set_couplings(bad)
    g.set_couplings(eps2)
    for kern in (lt.KERNEL_TILED, lt.KERNEL_RESIDENT):
        with pytest.raises(lt.LatticeError):
            g.set_kernel(kern)
    with pytest.raises(lt.LatticeError):
        g.set_dynamics(lt.DYNAMICS_RANDOM_SITE, 16, 16)
    g.close()
