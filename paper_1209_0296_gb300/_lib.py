"""ctypes binding of liblattice.so (argument marshalling only).

Every step of the sweep runs in the CUDA library; this module only converts
Python arguments to the C ABI of ``include/lattice.h`` and back.  If the
library has not been built, loading fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

c_int, c_int64, c_uint64, c_double, c_void_p, c_size_t = (
    ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t)


class LatticeRequest(ctypes.Structure):
    _fields_ = [("dims", c_int), ("L", c_int), ("two_S", c_int), ("model", c_int),
                ("J", c_double), ("h", c_double), ("T_or_c", c_double),
                ("seed", c_uint64), ("init", c_int), ("sweeps", c_int64), ("keep_spins", c_int)]


class LatticeResult(ctypes.Structure):
    _fields_ = [("status", c_int), ("sweeps_done", c_int64),
                ("bond", c_int64), ("mag", c_int64), ("up", c_int64), ("unflipped", c_int64),
                ("E", c_double), ("M", c_double), ("density", c_double), ("persistence", c_double),
                ("t_submit", c_double), ("t_admit", c_double), ("t_done", c_double)]


class LatticeStaticDesc(ctypes.Structure):
    _fields_ = [("L", c_int), ("J", c_double), ("h", c_double), ("T", c_double),
                ("seed", c_uint64), ("sweep0", c_int64), ("spins", c_void_p * 2),
                ("counters", c_void_p)]


# name -> (restype, argtypes)
SIGNATURES = {
    "lattice_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_int, c_int, c_int, c_double,
                               c_double, c_double, c_uint64, c_int, c_int, c_void_p]),
    "lattice_sweep": (c_int, [c_void_p, c_int64]),
    "lattice_observables": (c_int, [c_void_p] + [ctypes.POINTER(c_double)] * 4),
    "lattice_series": (c_int, [c_void_p, c_int64, c_int64] + [c_void_p] * 4),
    "lattice_set_reference": (c_int, [c_void_p, ctypes.POINTER(c_int64)]),
    "lattice_clear_reference": (c_int, [c_void_p]),
    "lattice_set_dynamics": (c_int, [c_void_p, c_int, c_int, c_int]),
    "lattice_set_couplings": (c_int, [c_void_p, c_void_p]),
    "lattice_set_fields": (c_int, [c_void_p, c_void_p]),
    "lattice_field_series": (c_int, [c_void_p, c_int64, c_int64, c_void_p]),
    "lattice_autocorrelation": (c_int, [c_void_p, c_int64, c_int64, ctypes.c_double, c_void_p, c_void_p]),
    "lattice_get_spins": (c_int, [c_void_p, c_void_p]),
    "lattice_set_spins": (c_int, [c_void_p, c_void_p]),
    "lattice_get_state": (c_int, [c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_int64)]),
    "lattice_set_state": (c_int, [c_void_p, c_void_p, c_void_p, c_int64]),
    "lattice_info": (c_int, [c_void_p] + [ctypes.POINTER(c_int64)] * 3),
    "lattice_device_spins": (c_int, [c_void_p, ctypes.POINTER(c_void_p), ctypes.POINTER(c_size_t)]),
    "lattice_set_kernel": (c_int, [c_void_p, c_int, c_int, c_int, c_int]),
    "lattice_get_kernel": (c_int, [c_void_p] + [ctypes.POINTER(c_int)] * 4),
    "lattice_threshold_table": (c_int, [c_int, c_int, c_int, c_double, c_double, c_double,
                                        c_void_p, c_void_p, c_int, ctypes.POINTER(c_int),
                                        ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    "lattice_synchronize": (c_int, [c_void_p]),
    "lattice_destroy": (None, [c_void_p]),
    "lattice_batch_create": (c_int, [ctypes.POINTER(c_void_p), c_void_p]),
    "lattice_batch_add": (c_int, [c_void_p, c_void_p, c_int64]),
    "lattice_batch_run": (c_int, [c_void_p]),
    "lattice_batch_tuning": (c_int, [c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "lattice_batch_synchronize": (c_int, [c_void_p]),
    "lattice_batch_destroy": (None, [c_void_p]),
    "lattice_server_create": (c_int, [ctypes.POINTER(c_void_p), c_size_t, c_int, c_int]),
    "lattice_server_submit": (c_int, [c_void_p, ctypes.POINTER(LatticeRequest),
                                      ctypes.POINTER(c_uint64)]),
    "lattice_server_poll": (c_int, [c_void_p, c_uint64, ctypes.POINTER(LatticeResult), c_void_p]),
    "lattice_server_drain": (c_int, [c_void_p, c_double]),
    "lattice_server_clock": (c_double, [c_void_p]),
    "lattice_server_stats": (c_int, [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_double), ctypes.POINTER(c_int64)]),
    "lattice_server_destroy": (None, [c_void_p]),
    "lattice_sweep_static": (c_int, [c_void_p, c_int, c_int64, c_void_p]),
    "lattice_strerror": (ctypes.c_char_p, [c_int]),
    "lattice_last_cuda_error": (ctypes.c_char_p, []),
    "lattice_version": (ctypes.c_char_p, []),
}

# Entry points outside include/lattice.h used only by the tests.
TEST_SIGNATURES = {
    "lattice_test_fail_alloc": (c_int, [c_int]),
}


def library_path() -> str:
    """liblattice.so in the package's build folder, or LATTICE_LIB if set."""
    return os.environ.get("LATTICE_LIB", _build.SO)


def load(build_if_missing: bool = True):
    """Load liblattice.so; build it first if it is missing and nvcc exists."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if path == _build.SO and (not os.path.exists(path) or not _build.up_to_date()):
            if not build_if_missing:
                raise RuntimeError("liblattice.so is not built: run __graft_entry__.build()")
            _build.build()
        lib = ctypes.CDLL(path)
        for name, (res, args) in {**SIGNATURES, **TEST_SIGNATURES}.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


class LatticeError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load()
        msg = lib.lattice_strerror(code).decode()
        if code == -3:
            msg += " (%s)" % lib.lattice_last_cuda_error().decode()
        super().__init__("%s: %s [%d]" % (where, msg, code))
        self.code = code


def check(code: int, where: str) -> int:
    if code < 0:
        raise LatticeError(code, where)
    return code
