"""Host-side checks of the C-ABI library (no GPU needed).

* liblattice.so loads and exports every entry point declared in
  include/lattice.h;
* the acceptance table the library builds on the host is bit-identical to
  the oracle's thresholds (§III.A: min[1, exp(-dH/T)]; §III.B c-mode rates);
* argument errors are reported before any GPU work.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1209_0296_gb300 as lt
from paper_1209_0296_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lattice.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lattice_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = lt.load()
    names = declared_functions()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the Python binding covers each of them with a signature
    assert set(names) <= set(_lib.SIGNATURES), set(names) - set(_lib.SIGNATURES)


def test_version_and_strerror():
    lib = lt.load()
    assert b"sm_103a" in lib.lattice_version()
    for code in range(0, -9, -1):
        assert lib.lattice_strerror(code) and lib.lattice_strerror(code) != b"unknown error"


TABLE_CASES = [
    (2, 1, lt.ISING, 1.0, 0.0, 2.269185),
    (2, 1, lt.ISING, 1.0, 0.0, 2.0),
    (2, 1, lt.ISING, 1.0, 0.0, 3.0),
    (2, 1, lt.ISING, -0.7, 0.35, 1.3),
    (3, 2, lt.ISING, 1.0, 0.0, 2.0 + 7 * 2.0 / 15),
    (3, 3, lt.ISING, 0.5, -0.2, 4.0),
    (3, 8, lt.ISING, 1.0, 0.1, 9.0),
    (2, 1, lt.NE, 0.0, 0.0, 0.05),
    (2, 1, lt.NE, 0.0, 0.0, 0.3),
    (2, 1, lt.NE, 0.0, 0.0, 0.8),
    (2, 1, lt.NE, 0.5, -1.0, 1.5),
]


@pytest.mark.parametrize("case", TABLE_CASES)
def test_threshold_table_matches_oracle(case):
    dims, two_S, model, J, h, Tc = case
    thr, alw, dsmax, nmax = lt.threshold_table(*case)
    nn = 2 * nmax + 1
    assert thr.size == (2 * dsmax + 1) * nn
    cmode = model == lt.NE and J == 0.0 and h == 0.0
    checked = 0
    for ds in range(-dsmax, dsmax + 1):
        if ds == 0:
            continue
        for n in range(-nmax, nmax + 1):
            k = (ds + dsmax) * nn + (n + nmax)
            if cmode:
                p = Tc / (1 - Tc) if ds > 0 else (1 - Tc) / Tc
                a, t = oracle.probability_threshold(p)
            else:
                a, t = oracle.metropolis_threshold(oracle.delta_energy(J, h, ds, n), Tc)
            assert bool(alw[k]) == a, (ds, n)
            if not a:
                assert int(thr[k]) == t, (ds, n, int(thr[k]), t)
            checked += 1
    assert checked > 10


@pytest.mark.parametrize("args", [
    (4, 16, 1, lt.ISING, 1.0, 0.0, 2.0, 1, lt.INIT_COLD, lt.INT8),      # dims
    (2, 15, 1, lt.ISING, 1.0, 0.0, 2.0, 1, lt.INIT_COLD, lt.INT8),      # odd L
    (2, 0, 1, lt.ISING, 1.0, 0.0, 2.0, 1, lt.INIT_COLD, lt.INT8),       # L < 2
    (2, 16, 0, lt.ISING, 1.0, 0.0, 2.0, 1, lt.INIT_COLD, lt.INT8),      # two_S
    (2, 16, 9, lt.ISING, 1.0, 0.0, 2.0, 1, lt.INIT_COLD, lt.INT8),      # two_S too large
    (3, 16, 1, lt.NE, 0.0, 0.0, 0.3, 1, lt.INIT_EQUILIBRIUM, lt.INT8),  # NE in 3D
    (2, 16, 2, lt.NE, 0.0, 0.0, 0.3, 1, lt.INIT_EQUILIBRIUM, lt.INT8),  # NE spin-1
    (2, 16, 1, lt.NE, 0.0, 0.0, 1.2, 1, lt.INIT_EQUILIBRIUM, lt.INT8),  # c out of range
    (2, 16, 1, lt.ISING, 1.0, 0.0, 0.0, 1, lt.INIT_COLD, lt.INT8),      # T = 0
    (2, 16, 1, lt.ISING, 1.0, 0.0, float("nan"), 1, lt.INIT_COLD, lt.INT8),
    (2, 16, 1, lt.ISING, 1.0, 0.0, 2.0, 1, lt.INIT_EQUILIBRIUM, lt.INT8),  # eq. init needs c-mode
    (2, 16, 1, lt.ISING, 1.0, 0.0, 2.0, 1, 7, lt.INT8),                 # init
    (2, 16, 1, lt.ISING, 1.0, 0.0, 2.0, 1, lt.INIT_COLD, 5),            # layout
    (3, 2048, 1, lt.ISING, 1.0, 0.0, 2.0, 1, lt.INIT_COLD, lt.INT8),    # N >= 2^32
])
def test_invalid_arguments_rejected_before_gpu_work(args):
    lib = lt.load()
    h = ctypes.c_void_p()
    rc = lib.lattice_create(ctypes.byref(h), *args, None)
    assert rc == -1, rc
    assert not h.value


def test_unsupported_layout_combination():
    lib = lt.load()
    h = ctypes.c_void_p()
    rc = lib.lattice_create(ctypes.byref(h), 3, 16, 1, lt.ISING, 1.0, 0.0, 2.0, 1, lt.INIT_COLD,
                            lt.BITPACKED, None)
    assert rc == -6


def test_null_handles_rejected():
    lib = lt.load()
    assert lib.lattice_sweep(None, 1) == -1
    assert lib.lattice_synchronize(None) == -1
    assert lib.lattice_get_spins(None, None) == -1
    lib.lattice_destroy(None)
    assert lib.lattice_threshold_table(2, 1, lt.ISING, 1.0, 0.0, -1.0, None, None, 0,
                                       None, None, None) == -1
