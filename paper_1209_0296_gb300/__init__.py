"""GB300 checkerboard spin-lattice sweeps (Levy, Cohen & Rabani, arXiv:1209.0296).

Python binding of the C-ABI CUDA library ``liblattice.so`` (``include/lattice.h``).
Same names as the C entry points; only argument marshalling happens here.
PyTorch is used only for streams (any object with a ``cuda_stream`` attribute,
or an integer ``cudaStream_t``).
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from ._lib import LatticeError, LatticeRequest, LatticeResult, check, load

__all__ = ["Lattice", "Batch", "Server", "LatticeError", "load", "threshold_table",
           "ISING", "NE", "POTTS", "INIT_COLD", "INIT_RANDOM", "INIT_EQUILIBRIUM", "INT8", "BITPACKED",
           "KERNEL_AUTO", "KERNEL_GENERIC", "KERNEL_TILED", "KERNEL_WIDE",
           "KERNEL_RESIDENT", "DYNAMICS_CHECKERBOARD", "DYNAMICS_RANDOM_SITE",
           "DYNAMICS_RANDOM_SITE_BALANCED"]

ISING, NE, POTTS = 0, 1, 2
INIT_COLD, INIT_RANDOM, INIT_EQUILIBRIUM = 0, 1, 2
INT8, BITPACKED = 0, 1
KERNEL_AUTO, KERNEL_GENERIC, KERNEL_TILED, KERNEL_WIDE, KERNEL_RESIDENT = 0, 1, 2, 3, 4
DYNAMICS_CHECKERBOARD, DYNAMICS_RANDOM_SITE, DYNAMICS_RANDOM_SITE_BALANCED = 0, 1, 2


def _stream_handle(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class Lattice:
    """One lattice resident on the GPU (``lattice_create`` ... ``lattice_destroy``)."""

    def __init__(self, dims=2, L=64, two_S=1, model=ISING, J=1.0, h=0.0, T_or_c=2.269185,
                 seed=0, init=INIT_COLD, layout=INT8, stream=None):
        self._lib = load()
        self.dims, self.L, self.two_S, self.model, self.layout = dims, L, two_S, model, layout
        self.J, self.h, self.T_or_c, self.seed = float(J), float(h), float(T_or_c), int(seed)
        self.N = L ** dims
        h_ = ctypes.c_void_p()
        check(self._lib.lattice_create(ctypes.byref(h_), dims, L, two_S, model, self.J, self.h,
                                       self.T_or_c, self.seed & (2**64 - 1), init, layout,
                                       _stream_handle(stream)), "lattice_create")
        self._h = h_

    @property
    def handle(self):
        return self._h

    def sweep(self, n: int):
        check(self._lib.lattice_sweep(self._h, int(n)), "lattice_sweep")

    def observables(self):
        v = [ctypes.c_double() for _ in range(4)]
        check(self._lib.lattice_observables(self._h, *[ctypes.byref(x) for x in v]),
              "lattice_observables")
        return dict(E=v[0].value, M=v[1].value, density=v[2].value, persistence=v[3].value)

    def series(self, first: int = 0, count: int | None = None):
        if count is None:
            count = self.sweeps() - first
        out = {k: np.zeros(count, dtype=np.int64) for k in ("bond", "mag", "up", "unflipped")}
        check(self._lib.lattice_series(self._h, int(first), int(count), _ptr(out["bond"]),
                                       _ptr(out["mag"]), _ptr(out["up"]), _ptr(out["unflipped"])),
              "lattice_series")
        return out

    def set_reference(self) -> int:
        """Store the current configuration as s(0) of the autocorrelation;
        returns the sweeps done at that moment."""
        r = ctypes.c_int64()
        check(self._lib.lattice_set_reference(self._h, ctypes.byref(r)), "lattice_set_reference")
        return r.value

    def set_couplings(self, bond_signs=None):
        """Per-bond coupling signs (dims*N int8 of +-1, bond_signs[d*N + i]
        for site i and its +e_d neighbour); None for uniform couplings."""
        if bond_signs is None:
            check(self._lib.lattice_set_couplings(self._h, None), "lattice_set_couplings")
            return
        a = np.ascontiguousarray(bond_signs, dtype=np.int8).reshape(-1)
        if a.size != self.dims * self.N:
            raise ValueError("need dims*N coupling signs")
        check(self._lib.lattice_set_couplings(self._h, _ptr(a)), "lattice_set_couplings")

    def set_fields(self, field_signs=None):
        """Per-site field signs eta_i = +-1 (N int8, x fastest; B_i = h *
        eta_i); None for the uniform field."""
        if field_signs is None:
            check(self._lib.lattice_set_fields(self._h, None), "lattice_set_fields")
            return
        a = np.ascontiguousarray(field_signs, dtype=np.int8).reshape(-1)
        if a.size != self.N:
            raise ValueError("need N field signs")
        check(self._lib.lattice_set_fields(self._h, _ptr(a)), "lattice_set_fields")

    def field_series(self, first: int, count: int | None = None):
        """Recorded sums sum_i eta_i s_i of sweeps [first, first+count)."""
        if count is None:
            count = self.sweeps() - first
        out = np.zeros(count, dtype=np.int64)
        check(self._lib.lattice_field_series(self._h, int(first), int(count), _ptr(out)),
              "lattice_field_series")
        return out

    def set_dynamics(self, dynamics=0, tile: int = 32, lam: int = 16):
        """DYNAMICS_CHECKERBOARD (default), DYNAMICS_RANDOM_SITE or
        DYNAMICS_RANDOM_SITE_BALANCED with tile x tile sub-lattices and lam
        picks per round."""
        check(self._lib.lattice_set_dynamics(self._h, int(dynamics), int(tile), int(lam)),
              "lattice_set_dynamics")

    def clear_reference(self):
        check(self._lib.lattice_clear_reference(self._h), "lattice_clear_reference")

    def autocorrelation(self, first: int, count: int | None = None, m: float | None = None):
        """Exact overlaps sum_i s_i(t) s_i(0) of sweeps [first, first+count)
        and Phi(t) with polarisation m (default 2c - 1 for a North-East
        lattice in c-mode; Phi omitted when m is unknown)."""
        if count is None:
            count = self.sweeps() - first
        ov = np.zeros(count, dtype=np.int64)
        own = m is None and self.model == NE and self.J == 0.0 and self.h == 0.0
        phi = np.zeros(count, dtype=np.float64) if (m is not None or own) else None
        check(self._lib.lattice_autocorrelation(self._h, int(first), int(count),
                                                math.nan if m is None else float(m), _ptr(ov), _ptr(phi)),
              "lattice_autocorrelation")
        return (ov, phi) if phi is not None else (ov, None)

    def get_spins(self, out=None):
        if out is None:
            out = np.empty(self.N, dtype=np.int8)
        check(self._lib.lattice_get_spins(self._h, _ptr(out)), "lattice_get_spins")
        return out

    def set_spins(self, spins):
        a = np.ascontiguousarray(spins, dtype=np.int8).reshape(-1)
        if a.size != self.N:
            raise ValueError("expected %d spins" % self.N)
        check(self._lib.lattice_set_spins(self._h, _ptr(a)), "lattice_set_spins")

    def get_state(self):
        s = np.empty(self.N, dtype=np.int8)
        f = np.empty(self.N, dtype=np.uint8)
        n = ctypes.c_int64()
        check(self._lib.lattice_get_state(self._h, _ptr(s), _ptr(f), ctypes.byref(n)),
              "lattice_get_state")
        return s, f, n.value

    def set_state(self, spins, flags=None, sweeps=0):
        s = np.ascontiguousarray(spins, dtype=np.int8).reshape(-1)
        f = None if flags is None else np.ascontiguousarray(flags, dtype=np.uint8).reshape(-1)
        check(self._lib.lattice_set_state(self._h, _ptr(s), _ptr(f), int(sweeps)),
              "lattice_set_state")

    def info(self):
        v = [ctypes.c_int64() for _ in range(3)]
        check(self._lib.lattice_info(self._h, *[ctypes.byref(x) for x in v]), "lattice_info")
        return dict(sweeps=v[0].value, n_sites=v[1].value, device_bytes=v[2].value)

    def sweeps(self) -> int:
        return self.info()["sweeps"]

    def device_spins(self):
        p = ctypes.c_void_p()
        n = ctypes.c_size_t()
        check(self._lib.lattice_device_spins(self._h, ctypes.byref(p), ctypes.byref(n)),
              "lattice_device_spins")
        return p.value, n.value

    def set_kernel(self, kernel=KERNEL_AUTO, tile_w=0, tile_h=0, sweeps_per_graph=0):
        check(self._lib.lattice_set_kernel(self._h, kernel, tile_w, tile_h, sweeps_per_graph),
              "lattice_set_kernel")

    def get_kernel(self):
        v = [ctypes.c_int() for _ in range(4)]
        check(self._lib.lattice_get_kernel(self._h, *[ctypes.byref(x) for x in v]),
              "lattice_get_kernel")
        return dict(kernel=v[0].value, tile_w=v[1].value, tile_h=v[2].value,
                    sweeps_per_graph=v[3].value)

    def sweeps_per_graph(self) -> int:
        return self.get_kernel()["sweeps_per_graph"]

    def tile_h(self) -> int:
        return self.get_kernel()["tile_h"]

    def set_spins_ptr(self, host_ptr: int):
        """lattice_set_spins from a raw host address holding N int8 spins (e.g. pinned memory)."""
        check(self._lib.lattice_set_spins(self._h, ctypes.c_void_p(host_ptr)), "lattice_set_spins")

    def series_into(self, first, count, bond=None, mag=None, up=None, unflipped=None):
        """lattice_series into caller-provided int64 arrays (no allocation)."""
        check(self._lib.lattice_series(self._h, int(first), int(count), _ptr(bond), _ptr(mag),
                                       _ptr(up), _ptr(unflipped)), "lattice_series")

    def threshold_table(self):
        return threshold_table(self.dims, self.two_S, self.model, self.J, self.h, self.T_or_c)

    def synchronize(self):
        check(self._lib.lattice_synchronize(self._h), "lattice_synchronize")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.lattice_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def threshold_table(dims, two_S, model, J, h, T_or_c):
    """Host-built acceptance table (``lattice_threshold_table``): (thr, always, dsmax, nmax)."""
    lib = load()
    cnt, dsmax, nmax = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    args = (int(dims), int(two_S), int(model), float(J), float(h), float(T_or_c))
    check(lib.lattice_threshold_table(*args, None, None, 0, ctypes.byref(cnt),
                                      ctypes.byref(dsmax), ctypes.byref(nmax)),
          "lattice_threshold_table")
    thr = np.zeros(cnt.value, dtype=np.uint32)
    alw = np.zeros(cnt.value, dtype=np.uint8)
    check(lib.lattice_threshold_table(*args, _ptr(thr), _ptr(alw), cnt.value, ctypes.byref(cnt),
                                      ctypes.byref(dsmax), ctypes.byref(nmax)),
          "lattice_threshold_table")
    return thr, alw, dsmax.value, nmax.value


class Batch:
    """Many lattices advanced together (``lattice_batch_*``)."""

    def __init__(self, stream=None):
        self._lib = load()
        h = ctypes.c_void_p()
        check(self._lib.lattice_batch_create(ctypes.byref(h), _stream_handle(stream)),
              "lattice_batch_create")
        self._h = h
        self._keep = []

    def add(self, lat: Lattice, n: int):
        check(self._lib.lattice_batch_add(self._h, lat.handle, int(n)), "lattice_batch_add")
        self._keep.append(lat)

    def run(self):
        check(self._lib.lattice_batch_run(self._h), "lattice_batch_run")
        self._keep = []

    def tuning(self):
        """Rows per 2D item (0 = size-based default) and steps per graph of the last run."""
        r, g = ctypes.c_int(), ctypes.c_int()
        check(self._lib.lattice_batch_tuning(self._h, ctypes.byref(r), ctypes.byref(g)), "lattice_batch_tuning")
        return dict(rows_per_item=r.value, steps_per_graph=g.value)

    def synchronize(self):
        check(self._lib.lattice_batch_synchronize(self._h), "lattice_batch_synchronize")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.lattice_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server of independent lattices (``lattice_server_*``)."""

    def __init__(self, hbm_budget_bytes=8 << 30, max_slots=1024, chunk_sweeps=256):
        self._lib = load()
        h = ctypes.c_void_p()
        check(self._lib.lattice_server_create(ctypes.byref(h), int(hbm_budget_bytes),
                                              int(max_slots), int(chunk_sweeps)),
              "lattice_server_create")
        self._h = h

    def submit(self, dims=2, L=64, two_S=1, model=ISING, J=1.0, h=0.0, T_or_c=2.269185, seed=0,
               init=INIT_RANDOM, sweeps=1000, keep_spins=False) -> int:
        req = LatticeRequest(dims, L, two_S, model, float(J), float(h), float(T_or_c),
                             int(seed) & (2**64 - 1), init, int(sweeps), 1 if keep_spins else 0)
        rid = ctypes.c_uint64()
        check(self._lib.lattice_server_submit(self._h, ctypes.byref(req), ctypes.byref(rid)),
              "lattice_server_submit")
        return rid.value

    def poll(self, rid: int, spins_out=None):
        """None while running; else a dict of the result (spins copied if requested)."""
        res = LatticeResult()
        rc = self._lib.lattice_server_poll(self._h, int(rid), ctypes.byref(res), _ptr(spins_out))
        if rc == -5:
            return None
        check(rc, "lattice_server_poll")
        return {k: getattr(res, k) for k, _ in LatticeResult._fields_}

    def drain(self, timeout_s: float = 0.0):
        check(self._lib.lattice_server_drain(self._h, float(timeout_s)), "lattice_server_drain")

    def clock(self) -> float:
        return self._lib.lattice_server_clock(self._h)

    def stats(self):
        """Device time of the rounds so far, the server's clock, rounds run."""
        busy, wall, rounds = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        check(self._lib.lattice_server_stats(self._h, ctypes.byref(busy), ctypes.byref(wall),
                                             ctypes.byref(rounds)), "lattice_server_stats")
        return dict(busy_s=busy.value, wall_s=wall.value, rounds=rounds.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.lattice_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
