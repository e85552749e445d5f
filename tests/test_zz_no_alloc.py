"""The no-allocation entry point, lattice_sweep_static.

Some callers cannot let a library allocate device memory: a framework whose
device memory all comes from its own caching pool, a memory-capped service,
or a caller that must not trigger the device-wide synchronisation an
allocation can cause.  lattice_sweep_static serves them: the caller passes
its own device buffers for the spins and the per-sweep counters, and the
library keeps its scratch in one fixed device array.  This test checks it,
through the C ABI, against the allocating entry points (lattice_create +
lattice_sweep) on two calls in a row: bit for bit, the tolerance of every
integer test here.  It sits in a file of its own that runs last.
"""
import ctypes

import numpy as np
import pytest

import paper_1209_0296_gb300 as lt
from paper_1209_0296_gb300 import _lib

pytestmark = pytest.mark.gpu

CASES = [  # L, J, h, T, seed
    (64, 1.0, 0.0, 2.269185, 1234),
    (96, 0.8, 0.2, 2.5, 7),
    (256, 1.0, 0.0, 3.0, 11),
]


def to_planar(lin, L):
    """x-fastest spins -> checkerboard planes: plane c, row y holds x = 2j + ((c+y) & 1)."""
    s = lin.reshape(L, L)
    out = np.empty((2, L, L // 2), dtype=np.int8)
    for y in range(L):
        for c in (0, 1):
            out[c, y] = s[y, ((c + y) & 1)::2]
    return out.reshape(-1)


def to_linear(pl, L):
    p = pl.reshape(2, L, L // 2)
    s = np.empty((L, L), dtype=np.int8)
    for y in range(L):
        for c in (0, 1):
            s[y, ((c + y) & 1)::2] = p[c, y]
    return s.reshape(-1)


def _descs(cases, bufs, counters, sweep0):
    arr = (_lib.LatticeStaticDesc * len(cases))()
    for i, (L, J, h, T, seed) in enumerate(cases):
        d = arr[i]
        d.L, d.J, d.h, d.T, d.seed, d.sweep0 = L, J, h, T, seed, sweep0
        d.spins[0] = bufs[i][0].data_ptr()
        d.spins[1] = bufs[i][1].data_ptr()
        d.counters = counters[i].data_ptr()
    return arr


def _two_calls_match(cases, n1=7, n2=5):
    """Two lattice_sweep_static calls in a row against lattice_create +
    lattice_sweep of the same lattices: spins and counters bit for bit."""
    torch = pytest.importorskip("torch")
    lib = lt.load()
    dev = torch.device("cuda", 0)
    refs = [lt.Lattice(2, L, 1, lt.ISING, J, h, T, seed=s, init=lt.INIT_RANDOM)
            for (L, J, h, T, s) in cases]
    bufs = []
    for g, (L, *_rest) in zip(refs, cases):
        b = torch.empty((2, L * L), dtype=torch.int8, device=dev)
        b[0].copy_(torch.from_numpy(to_planar(g.get_spins(), L)).to(dev))
        bufs.append(b)
    stream = torch.cuda.current_stream(dev).cuda_stream
    # first call: sweeps 0 .. n1-1
    c1 = [torch.zeros(4 * n1, dtype=torch.int64, device=dev) for _ in cases]
    rc = lib.lattice_sweep_static(ctypes.cast(_descs(cases, bufs, c1, 0), ctypes.c_void_p), len(cases), n1,
                                  ctypes.c_void_p(stream))
    assert rc == 0, lib.lattice_strerror(rc)
    torch.cuda.synchronize(dev)
    for g in refs:
        g.sweep(n1)
    for i, ((L, *_rest), g) in enumerate(zip(cases, refs)):
        ser = g.series(0, n1)
        got = c1[i].view(n1, 4).cpu().numpy()
        assert np.array_equal(got[:, 0], ser["bond"]) and np.array_equal(got[:, 1], ser["mag"])
        assert np.array_equal(got[:, 2], ser["up"])
        assert np.array_equal(to_linear(bufs[i][n1 & 1].cpu().numpy(), L), g.get_spins())
    # second call continues the same chains: sweeps n1 .. n1+n2-1
    c2 = [torch.full((4 * n2,), 123, dtype=torch.int64, device=dev) for _ in cases]  # cleared by the call
    rc = lib.lattice_sweep_static(ctypes.cast(_descs(cases, bufs, c2, n1), ctypes.c_void_p), len(cases), n2,
                                  ctypes.c_void_p(stream))
    assert rc == 0, lib.lattice_strerror(rc)
    torch.cuda.synchronize(dev)
    for g in refs:
        g.sweep(n2)
    for i, ((L, *_rest), g) in enumerate(zip(cases, refs)):
        ser = g.series(n1, n2)
        got = c2[i].view(n2, 4).cpu().numpy()
        assert np.array_equal(got[:, 0], ser["bond"]) and np.array_equal(got[:, 1], ser["mag"])
        assert np.array_equal(got[:, 2], ser["up"]) and np.all(got[:, 3] == 0)
        assert np.array_equal(to_linear(bufs[i][(n1 + n2) & 1].cpu().numpy(), L), g.get_spins())
    for g in refs:
        g.close()


def test_static_sweep_matches_allocating_entry_points_on_two_calls():
    _two_calls_match(CASES)


def test_static_sweep_at_the_lattice_limit():
    # 64 lattices (the most one call takes) of L = 32, each a single ragged tile
    _two_calls_match([(32, 1.0, 0.0, 2.0 + 0.02 * i, 100 + i) for i in range(64)], n1=4, n2=3)


def test_static_sweep_ragged_tiles():
    # L = 1056: 4 full tile columns and a ragged one, 16 full tile rows and a
    # ragged one, beside a lattice of whole tiles
    _two_calls_match([(1056, 1.0, 0.0, 2.269185, 5), (512, 1.0, 0.1, 2.4, 6)], n1=3, n2=2)


def test_static_sweep_rejects_sizes_beyond_its_limits():
    lib = lt.load()
    dummy = ctypes.c_void_p(256)   # never dereferenced: every check precedes GPU work

    def call(Ls, n=1):
        arr = (_lib.LatticeStaticDesc * len(Ls))()
        for d, L in zip(arr, Ls):
            d.L, d.J, d.h, d.T, d.seed, d.sweep0 = L, 1.0, 0.0, 2.5, 1, 0
            d.spins[0] = d.spins[1] = dummy.value
            d.counters = dummy.value
        return lib.lattice_sweep_static(ctypes.cast(arr, ctypes.c_void_p), len(Ls), n, None)

    assert call([32768, 32768]) == -7          # 131072 tiles > 65536
    assert call([64] * 65) == -7               # more than 64 lattices
    assert call([48]) == -6                    # L not a multiple of 32
    assert call([63]) == -1                    # odd L
    assert lib.lattice_sweep_static(None, 1, 1, None) == -1
