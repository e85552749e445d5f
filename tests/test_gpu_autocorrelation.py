"""Spin-spin autocorrelation on the GPU (§III.B, Eq. 4): the
per-sweep overlap sum_i s_i(t) s_i(0) recorded inside every sweep kernel
must equal the oracle's, integer for integer, for every kernel, layout and
model, in the batched engine too; Phi follows from it on the host."""
import numpy as np
import pytest

import oracle
import paper_1209_0296_gb300 as lt

pytestmark = pytest.mark.gpu


def pair(dims, L, two_S, model, J, h, Tc, seed, init, pre, n, kernel=lt.KERNEL_AUTO,
         layout=lt.INT8, chunks=None):
    o = oracle.Lattice(dims, L, two_S, model, J, h, Tc, seed=seed, init=init)
    g = lt.Lattice(dims, L, two_S, model, J, h, Tc, seed=seed, init=init, layout=layout)
    try:
        if layout == lt.INT8:
            g.set_kernel(kernel)
        o.sweep(pre)
        g.sweep(pre)
        assert g.set_reference() == pre
        o.set_reference()
        ser_o = o.sweep(n)
        for c in (chunks or [n]):
            g.sweep(c)
        ov, _ = g.autocorrelation(pre, n, m=0.0)
        assert np.array_equal(ov, ser_o["overlap"])
        assert np.array_equal(g.get_spins(), o.spins)
        ser = g.series(pre, n)
        for k in ("bond", "mag", "up"):
            assert np.array_equal(ser[k], ser_o[k]), k
        return ov
    finally:
        g.close()


@pytest.mark.parametrize("kernel", [lt.KERNEL_GENERIC, lt.KERNEL_TILED, lt.KERNEL_WIDE,
                                    lt.KERNEL_RESIDENT, lt.KERNEL_AUTO])
@pytest.mark.parametrize("L", [64, 96, 128])
def test_ising_2d_every_kernel(kernel, L):
    pair(2, L, 1, lt.ISING, 1.0, 0.05, 2.4, 50 + L, lt.INIT_RANDOM, 5, 30, kernel=kernel,
         chunks=[1, 11, 18])


@pytest.mark.parametrize("kernel", [lt.KERNEL_GENERIC, lt.KERNEL_TILED, lt.KERNEL_WIDE,
                                    lt.KERNEL_RESIDENT])
def test_north_east_every_kernel_and_phi(kernel):
    c = 0.2
    L = 96
    o = oracle.Lattice(2, L, 1, lt.NE, 0.0, 0.0, c, seed=3, init=lt.INIT_EQUILIBRIUM)
    g = lt.Lattice(2, L, 1, lt.NE, 0.0, 0.0, c, seed=3, init=lt.INIT_EQUILIBRIUM)
    g.set_kernel(kernel)
    g.set_reference()
    o.set_reference()
    ser_o = o.sweep(40)
    g.sweep(40)
    ov, phi = g.autocorrelation(0, 40)
    assert np.array_equal(ov, ser_o["overlap"])
    m = 2 * c - 1
    assert np.allclose(phi, (ov / g.N - m * m) / (1 - m * m), rtol=0, atol=1e-15)
    g.close()


@pytest.mark.parametrize("model,Tc,init", [(lt.ISING, 2.269185, lt.INIT_RANDOM),
                                           (lt.NE, 0.3, lt.INIT_EQUILIBRIUM)])
def test_bitpacked_layout(model, Tc, init):
    J = 1.0 if model == lt.ISING else 0.0
    pair(2, 128, 1, model, J, 0.0, Tc, 8, init, 3, 25, layout=lt.BITPACKED)


@pytest.mark.parametrize("dims,L,two_S", [(3, 16, 1), (3, 32, 2), (2, 48, 3), (3, 10, 2), (2, 22, 1)])
def test_three_d_spin_S_and_generic_sizes(dims, L, two_S):
    # wide 3D/spin-S kernel (L % 16 == 0) and the generic kernel (other L)
    pair(dims, L, two_S, lt.ISING, 1.0, 0.1, 2.5 * two_S, 30 + L, lt.INIT_RANDOM, 2, 20)


def test_free_spins_closed_form_on_the_gpu():
    # J = h = 0: every spin flips every sweep, overlap = (-1)^t N
    g = lt.Lattice(2, 128, 1, lt.ISING, 0.0, 0.0, 1.0, seed=1, init=lt.INIT_RANDOM)
    g.set_reference()
    g.sweep(12)
    ov, _ = g.autocorrelation(0, 12)
    assert list(ov) == [(-1) ** t * g.N for t in range(1, 13)]
    g.close()


def test_reference_taken_after_graphs_were_captured():
    # graph-replayed sweeps before and after the reference is set: the
    # replayed graphs must pick up the new descriptor
    o = oracle.Lattice(2, 256, 1, lt.ISING, 1.0, 0.0, 2.3, seed=12, init=lt.INIT_RANDOM)
    g = lt.Lattice(2, 256, 1, lt.ISING, 1.0, 0.0, 2.3, seed=12, init=lt.INIT_RANDOM)
    g.set_kernel(lt.KERNEL_WIDE, 0, 0, 8)
    o.sweep(40)
    g.sweep(40)
    g.set_reference()
    o.set_reference()
    ser_o = o.sweep(50)
    g.sweep(50)
    ov, _ = g.autocorrelation(40, 50)
    assert np.array_equal(ov, ser_o["overlap"])
    # a second reference replaces the first
    g.set_reference()
    o.set_reference()
    ser_o = o.sweep(17)
    g.sweep(17)
    ov, _ = g.autocorrelation(90, 17)
    assert np.array_equal(ov, ser_o["overlap"])
    g.close()


def test_reference_errors():
    g = lt.Lattice(2, 64, 1, lt.ISING, 1.0, 0.0, 2.0, seed=1, init=lt.INIT_RANDOM)
    g.sweep(3)
    with pytest.raises(lt.LatticeError):
        g.autocorrelation(0, 3)          # no reference yet
    g.set_reference()
    g.sweep(4)
    with pytest.raises(lt.LatticeError):
        g.autocorrelation(2, 3)          # before the reference
    with pytest.raises(lt.LatticeError):
        g.autocorrelation(3, 5)          # past the last sweep
    with pytest.raises(lt.LatticeError):
        g.autocorrelation(3, 4, m=1.0)   # |m| must be < 1
    ov, _ = g.autocorrelation(3, 4, m=0.0)
    assert ov.shape == (4,)
    g.clear_reference()
    with pytest.raises(lt.LatticeError):
        g.autocorrelation(3, 4)
    g.sweep(5)                           # sweeps go on without a reference
    g.close()


def test_batched_lattices_with_references():
    cfgs = [(2, 288, 1, lt.ISING, 1.0, 0.0, 2.3, 61, lt.INIT_RANDOM),     # tiled items
            (2, 64, 1, lt.NE, 0.0, 0.0, 0.25, 62, lt.INIT_EQUILIBRIUM),   # resident CTA
            (3, 16, 2, lt.ISING, 1.0, 0.0, 3.3, 63, lt.INIT_RANDOM),      # wide 3D items
            (3, 6, 1, lt.ISING, 1.0, 0.0, 4.0, 64, lt.INIT_RANDOM),       # generic chunks
            (3, 32, 1, lt.ISING, 1.0, 0.0, 4.3, 66, lt.INIT_RANDOM),      # byte-parallel 3D spin-1/2
            (2, 48, 2, lt.ISING, 1.0, 0.1, 1.8, 67, lt.INIT_RANDOM),      # byte-parallel 2D spin-1
            (3, 16, 3, lt.ISING, 1.0, 0.0, 8.0, 68, lt.INIT_RANDOM),      # per-site 3D items
            (3, 16, 2, lt.ISING, 1.0, 0.0, 0.25, 69, lt.INIT_RANDOM),     # per site: never-accept entries
            (2, 64, 1, lt.ISING, 1.0, 0.0, 2.3, 65, lt.INIT_RANDOM)]      # no reference
    lats = [lt.Lattice(*c[:7], seed=c[7], init=c[8]) for c in cfgs]
    ors = [oracle.Lattice(*c[:7], seed=c[7], init=c[8]) for c in cfgs]
    for g, o in zip(lats[:-1], ors[:-1]):
        g.sweep(2)
        o.sweep(2)
        g.set_reference()
        o.set_reference()
    b = lt.Batch()
    for g in lats:
        b.add(g, 37)
    b.run()
    b.synchronize()
    for g, o in zip(lats[:-1], ors[:-1]):
        ser_o = o.sweep(37)
        ov, _ = g.autocorrelation(2, 37, m=0.0)
        assert np.array_equal(ov, ser_o["overlap"])
        assert np.array_equal(g.get_spins(), o.spins)
    with pytest.raises(lt.LatticeError):
        lats[-1].autocorrelation(0, 37)
    b.close()


@pytest.mark.slow
def test_full_size_north_east_L8192_reference():
    # North-East L = 8192, c = 0.3, equilibrium start (seed 21): overlap of
    # the first two sweeps with the initial state
    pair(2, 8192, 1, lt.NE, 0.0, 0.0, 0.3, 21, lt.INIT_EQUILIBRIUM, 0, 2)


def test_default_polarisation_is_the_models_own():
    # m = NaN (the binding's m=None) asks the library for the North-East
    # model's own polarisation, <s_i> = 2c - 1 (Eq. 4): the same Phi as an
    # explicit m; a lattice without one refuses Phi but still gives overlaps
    c = 0.3
    g = lt.Lattice(2, 64, 1, lt.NE, 0.0, 0.0, c, seed=21, init=lt.INIT_EQUILIBRIUM)
    g.set_reference()
    g.sweep(12)
    ov_d, phi_d = g.autocorrelation(0, 12)
    ov_e, phi_e = g.autocorrelation(0, 12, m=2 * c - 1)
    assert np.array_equal(ov_d, ov_e)
    assert np.allclose(phi_d, phi_e, rtol=0, atol=1e-15)
    g.close()
    h = lt.Lattice(2, 64, 1, lt.ISING, 1.0, 0.0, 2.5, seed=3, init=lt.INIT_RANDOM)
    h.set_reference()
    h.sweep(5)
    ov, phi = h.autocorrelation(0, 5)
    assert phi is None and ov.shape == (5,)
    h.close()
