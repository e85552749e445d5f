"""CPU oracle for the checkerboard spin-lattice sweep -- TEST INFRASTRUCTURE ONLY.

A plain single-threaded restatement (``oracle.c``) of the checkerboard
Metropolis sweep for spin-S Ising models (Levy, Cohen & Rabani, §III.A,
Eq. 2) and of the facilitated North-East sweep (§III.B, Eq. 3), used to check
the CUDA library bit for bit.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU baseline may import this package; the library never
does, and the two share no code.

Parity pins: see the ``-m "not gpu"`` tests in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ISING, NE, POTTS = 0, 1, 2
INIT_COLD, INIT_RANDOM, INIT_EQUILIBRIUM = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared object with gcc (no GPU needed)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i8p = np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")
            u8p = ctypes.c_void_p
            i64p = ctypes.c_void_p
            u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
            lib.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
            lib.oracle_philox4x32_10.restype = None
            lib.oracle_init.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_uint64, ctypes.c_int, i8p]
            lib.oracle_init.restype = ctypes.c_int
            lib.oracle_sweep.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_uint64, i8p, u8p, ctypes.c_int64,
                                         ctypes.c_int64, i64p, i64p, i64p, i64p]
            lib.oracle_sweep.restype = ctypes.c_int
            lib.oracle_measure.argtypes = [ctypes.c_int, ctypes.c_int, i8p, u8p,
                                           i64p, i64p, i64p, i64p]
            lib.oracle_measure.restype = None
            lib.oracle_rsite_sweep.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                               ctypes.c_int, ctypes.c_int, i8p, ctypes.c_void_p,
                                               ctypes.c_int64, ctypes.c_int64] + [ctypes.c_void_p] * 4
            lib.oracle_rsite_sweep.restype = ctypes.c_int
            lib.oracle_rsite_sweep_variant.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                       ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                                       ctypes.c_int, ctypes.c_int, ctypes.c_int, i8p,
                                                       ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64] + \
                [ctypes.c_void_p] * 4
            lib.oracle_rsite_sweep_variant.restype = ctypes.c_int
            lib.oracle_sweep_couplings.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                   ctypes.c_uint64, i8p, ctypes.c_void_p, ctypes.c_void_p,
                                                   ctypes.c_int64, ctypes.c_int64] + [ctypes.c_void_p] * 4
            lib.oracle_sweep_couplings.restype = ctypes.c_int
            lib.oracle_sweep_disorder.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_uint64, i8p, ctypes.c_void_p, ctypes.c_void_p,
                                                  ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64] + \
                [ctypes.c_void_p] * 5
            lib.oracle_sweep_disorder.restype = ctypes.c_int
            lib.oracle_measure_disorder.argtypes = [ctypes.c_int, ctypes.c_int, i8p, ctypes.c_void_p,
                                                    ctypes.c_void_p, ctypes.c_void_p] + \
                [ctypes.POINTER(ctypes.c_int64)] * 5
            lib.oracle_measure_disorder.restype = None
            lib.oracle_measure_couplings.argtypes = [ctypes.c_int, ctypes.c_int, i8p, ctypes.c_void_p,
                                                     ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int64)] * 4
            lib.oracle_measure_couplings.restype = None
            lib.oracle_measure_potts.argtypes = [ctypes.c_int, ctypes.c_int, i8p] + \
                [ctypes.POINTER(ctypes.c_int64)] * 3
            lib.oracle_measure_potts.restype = None
            lib.oracle_overlap.argtypes = [ctypes.c_int64, i8p, i8p]
            lib.oracle_overlap.restype = ctypes.c_int64
            lib.oracle_overlap_potts.argtypes = [ctypes.c_int64, i8p, i8p]
            lib.oracle_overlap_potts.restype = ctypes.c_int64
            lib.oracle_metropolis_threshold.argtypes = [ctypes.c_double, ctypes.c_double,
                                                        ctypes.POINTER(ctypes.c_uint32)]
            lib.oracle_metropolis_threshold.restype = ctypes.c_int
            lib.oracle_probability_threshold.argtypes = [ctypes.c_double,
                                                         ctypes.POINTER(ctypes.c_uint32)]
            lib.oracle_probability_threshold.restype = ctypes.c_int
            lib.oracle_delta_energy.argtypes = [ctypes.c_double, ctypes.c_double,
                                                ctypes.c_int, ctypes.c_int]
            lib.oracle_delta_energy.restype = ctypes.c_double
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(counter, key):
    """Philox4x32-10 (Salmon et al., SC'11) of one 4-word counter and 2-word key."""
    lib = _load()
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.oracle_philox4x32_10(c, k, out)
    return out


def metropolis_threshold(dE: float, T: float):
    """(always, thr): Metropolis acceptance min[1, exp(-dE/T)] as an integer threshold."""
    lib = _load()
    thr = ctypes.c_uint32(0)
    always = lib.oracle_metropolis_threshold(float(dE), float(T), ctypes.byref(thr))
    return bool(always), int(thr.value)


def probability_threshold(p: float):
    lib = _load()
    thr = ctypes.c_uint32(0)
    always = lib.oracle_probability_threshold(float(p), ctypes.byref(thr))
    return bool(always), int(thr.value)


def delta_energy(J: float, h: float, ds: int, n: int) -> float:
    return _load().oracle_delta_energy(float(J), float(h), int(ds), int(n))


class Lattice:
    """A lattice advanced by the oracle: spins (int8, x fastest) + persistence flags."""

    def __init__(self, dims, L, two_S=1, model=ISING, J=1.0, h=0.0, T_or_c=2.269185,
                 seed=0, init=INIT_COLD):
        self.dims, self.L, self.two_S, self.model = dims, L, two_S, model
        self.J, self.h, self.T_or_c, self.seed = float(J), float(h), float(T_or_c), int(seed)
        self.N = L ** dims
        self.spins = np.zeros(self.N, dtype=np.int8)
        self.flags = np.zeros(self.N, dtype=np.uint8)
        self.sweep_index = 0
        self.ref = None          # s(0) of the autocorrelation (§III.B, Phi(t))
        self.eps = None          # per-bond signs (Eq. 1 couplings J_ij = J * eps), or None
        self.eta = None          # per-site field signs (Eq. 1 fields B_i = h * eta), or None
        rc = _load().oracle_init(dims, L, two_S, model, self.J, self.h, self.T_or_c,
                                 self.seed, init, self.spins)
        if rc != 0:
            raise ValueError("oracle_init rejected the parameters")

    def set_couplings(self, eps):
        """Per-bond signs: eps[d*N + i] = +-1 for the bond from linear site i
        to its +e_d neighbour (Eq. 1 with J_ij = J * eps); None for uniform."""
        if eps is None:
            self.eps = None
            return
        e = np.ascontiguousarray(eps, dtype=np.int8).reshape(-1)
        if e.size != self.dims * self.N or not np.all(np.abs(e) == 1):
            raise ValueError("couplings must be dims*N values of +-1")
        self.eps = e

    def set_fields(self, eta):
        """Per-site field signs eta_i = +-1 (B_i = h * eta_i); None for uniform."""
        if eta is None:
            self.eta = None
            return
        e = np.ascontiguousarray(eta, dtype=np.int8).reshape(-1)
        if e.size != self.N or not np.all(np.abs(e) == 1):
            raise ValueError("fields must be N values of +-1")
        self.eta = e

    def set_reference(self):
        """Take the current configuration as s(0) of the autocorrelation."""
        self.ref = self.spins.copy()

    def overlap(self):
        """sum_i s_i * s_i(0) of the current configuration (needs a reference);
        for the Potts model the number of sites with s_i = s_i(0)."""
        if self.model == POTTS:
            return int(_load().oracle_overlap_potts(self.N, self.spins, self.ref))
        return int(_load().oracle_overlap(self.N, self.spins, self.ref))

    def sweep(self, n: int):
        """Advance n sweeps; returns dict of per-sweep int64 series (bond, mag, up,
        unflipped, and "overlap" = sum_i s_i(t) s_i(0) when a reference is set)."""
        if self.ref is not None:
            keys = ("bond", "mag", "up", "unflipped", "field")
            out = {k: np.zeros(n, dtype=np.int64) for k in keys + ("overlap",)}
            for k in range(n):      # one sweep at a time, the overlap after each
                one = self._sweep(1)
                for key in keys:
                    out[key][k] = one[key][0]
                out["overlap"][k] = self.overlap()
            return out
        return self._sweep(n)

    def rsite_sweep(self, n: int, tile: int, lam: int, balanced: bool = False):
        """Advance n sweeps of the paper's random-sub-lattice, random-site
        algorithm (§III.B) with b x b sub-lattices and lam picks per round
        (balanced: its balance-preserving variant, single-colour rounds and
        four launches per sweep); returns the per-sweep series (and
        "overlap" when a reference is set)."""
        keys = ("bond", "mag", "up", "unflipped")
        if self.ref is not None:
            out = {k: np.zeros(n, dtype=np.int64) for k in keys + ("overlap",)}
            for k in range(n):
                one = self._rsite(1, tile, lam, balanced)
                for key in keys:
                    out[key][k] = one[key][0]
                out["overlap"][k] = self.overlap()
            return out
        return self._rsite(n, tile, lam, balanced)

    def _rsite(self, n, tile, lam, balanced=False):
        if self.dims != 2 or self.two_S != 1 or self.eps is not None or self.eta is not None:
            raise ValueError("the random-site algorithm is 2D spin-1/2 with uniform couplings")
        out = {k: np.zeros(n, dtype=np.int64) for k in ("bond", "mag", "up", "unflipped")}
        rc = _load().oracle_rsite_sweep_variant(self.L, self.model, self.J, self.h, self.T_or_c, self.seed,
                                                int(tile), int(lam), int(bool(balanced)), self.spins,
                                                _ptr(self.flags) if self.model == NE else None,
                                                self.sweep_index, n, _ptr(out["bond"]), _ptr(out["mag"]),
                                                _ptr(out["up"]), _ptr(out["unflipped"]))
        if rc != 0:
            raise ValueError("oracle_rsite_sweep rejected the parameters")
        self.sweep_index += n
        return out

    def _sweep(self, n: int):
        """Series also carry "field" = sum_i eta_i s_i (= mag without field signs)."""
        out = {k: np.zeros(n, dtype=np.int64) for k in ("bond", "mag", "up", "unflipped", "field")}
        rc = _load().oracle_sweep_disorder(self.dims, self.L, self.two_S, self.model, self.J, self.h,
                                           self.T_or_c, self.seed, self.spins,
                                           _ptr(self.flags) if self.model == NE else None,
                                           _ptr(self.eps), _ptr(self.eta), self.sweep_index, n,
                                           _ptr(out["bond"]), _ptr(out["mag"]), _ptr(out["up"]),
                                           _ptr(out["unflipped"]), _ptr(out["field"]))
        if rc != 0:
            raise ValueError("oracle_sweep rejected the parameters")
        self.sweep_index += n
        return out

    def measure(self):
        b, m, u, f = (ctypes.c_int64() for _ in range(4))
        if self.model == POTTS:
            _load().oracle_measure_potts(self.dims, self.L, self.spins, ctypes.byref(b), ctypes.byref(m),
                                         ctypes.byref(u))
            return dict(bond=b.value, mag=m.value, up=u.value, unflipped=0)
        fs = ctypes.c_int64()
        _load().oracle_measure_disorder(self.dims, self.L, self.spins,
                                        _ptr(self.flags) if self.model == NE else None, _ptr(self.eps),
                                        _ptr(self.eta), ctypes.byref(b), ctypes.byref(m), ctypes.byref(u),
                                        ctypes.byref(f), ctypes.byref(fs))
        return dict(bond=b.value, mag=m.value, up=u.value, unflipped=f.value, field=fs.value)

    def energy(self, bond, mag):
        """E = -J*bond - h*mag; with field signs pass the series' "field" as mag."""
        J, h = self.J, self.h
        if self.model == NE and J == 0.0 and h == 0.0:
            J, h = 0.0, -1.0
        return -J * np.asarray(bond, dtype=np.float64) - h * np.asarray(mag, dtype=np.float64)
