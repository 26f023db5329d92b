"""ctypes loader of the CUDA library ``libparcels_gb.so`` (argument marshalling only).

The library is built in-tree by :mod:`paper_1707_05163_gb300.build`.  There is
no fallback: if the shared library is missing or cannot be loaded, every call
raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

PG_OK = 0
PG_ERR_ARG, PG_ERR_CUDA, PG_ERR_STATE, PG_ERR_TIME = -1, -2, -3, -4
PG_ERR_CALLBACK, PG_ERR_TIMEOUT, PG_ERR_NOMEM, PG_ERR_UNSUPPORTED, PG_ERR_DEVICE = -5, -6, -7, -8, -9
PG_FLAT, PG_SPHERICAL = 0, 1
PG_F64, PG_F32, PG_F16S, PG_BF16S = 0, 1, 2, 3
PG_POS_F64, PG_POS_F32, PG_POS_CELL = 0, 1, 2
PG_EULER, PG_RK4, PG_RKF45 = 0, 1, 2
PG_BROWNIAN, PG_SINK, PG_SETTLE, PG_AGE, PG_SAMPLE = 1, 2, 4, 8, 16
PG_LINEAR, PG_NEAREST = 0, 1
PG_ALIVE, PG_OOB_HORIZ, PG_OOB_DEPTH, PG_NAN, PG_DELETED = 0, 1, 2, 3, 4

ERROR_NAMES = {
    -1: "PG_ERR_ARG", -2: "PG_ERR_CUDA", -3: "PG_ERR_STATE", -4: "PG_ERR_TIME",
    -5: "PG_ERR_CALLBACK", -6: "PG_ERR_TIMEOUT", -7: "PG_ERR_NOMEM", -8: "PG_ERR_UNSUPPORTED",
    -9: "PG_ERR_DEVICE",
}


class PGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("lon", C.c_void_p), ("lat", C.c_void_p), ("depth", C.c_void_p)]


class Tune(C.Structure):
    _fields_ = [("block", C.c_int), ("resort_steps", C.c_int), ("chunk_steps", C.c_int)]


class SurrogateStats(C.Structure):
    _fields_ = [("network_steps", C.c_int64), ("checked", C.c_int64), ("rejected", C.c_int64),
                ("rk4_particle_steps", C.c_int64), ("error_sum", C.c_double),
                ("seconds_network", C.c_double), ("seconds_rk4", C.c_double),
                ("seconds_total", C.c_double)]


SNAPSHOT_CB = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_size_t)
OUTPUT_CB = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_double, C.c_int64, C.c_void_p, C.c_void_p,
                        C.c_void_p, C.c_void_p, C.c_void_p)

class Record(C.Structure):
    _fields_ = [("time", C.c_double), ("n", C.c_int64), ("nvar", C.c_int),
                ("var_stride", C.c_int64), ("id", C.c_void_p), ("lon", C.c_void_p),
                ("lat", C.c_void_p), ("depth", C.c_void_p), ("status", C.c_void_p),
                ("age", C.c_void_p), ("vars", C.c_void_p)]


RECORD_CB = C.CFUNCTYPE(C.c_int, C.c_void_p, C.POINTER(Record))

_P = C.c_void_p
_SIGS = {
    "pg_last_error": ([], C.c_char_p),
    "pg_version": ([], C.c_char_p),
    "pg_fieldset_create": ([C.POINTER(Grid), C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(_P)],
                           C.c_int),
    "pg_fieldset_set_times": ([_P, C.c_int, _P, C.c_double], C.c_int),
    "pg_fieldset_load_snapshot": ([_P, C.c_int, _P, C.c_int, _P], C.c_int),
    "pg_fieldset_stream": ([_P, _P, SNAPSHOT_CB, _P, C.c_int], C.c_int),
    "pg_fieldset_device_bytes": ([_P, C.POINTER(C.c_size_t)], C.c_int),
    "pg_fieldset_set_ring": ([_P, C.c_int], C.c_int),
    "pg_fieldset_get_scale": ([_P, C.c_int, C.c_int, C.POINTER(C.c_float)], C.c_int),
    "pg_fieldset_destroy": ([_P], C.c_int),
    "pg_fieldset_add_constant": ([_P, C.c_char_p, C.c_double], C.c_int),
    "pg_fieldset_get_constant": ([_P, C.c_char_p, C.POINTER(C.c_double)], C.c_int),
    "pg_fieldset_set_interp": ([_P, C.c_int], C.c_int),
    "pg_fieldset_add_scalar": ([_P, C.c_char_p, C.c_int, C.POINTER(C.c_int)], C.c_int),
    "pg_fieldset_load_scalar": ([_P, C.c_int, C.c_int, _P, C.c_int, _P], C.c_int),
    "pg_pset_get_variables": ([_P, _P, _P, _P], C.c_int),
    "pg_kernel_create": ([C.c_int, C.c_uint, C.c_double, C.c_double, C.POINTER(_P)], C.c_int),
    "pg_kernel_destroy": ([_P], C.c_int),
    "pg_pset_create": ([_P, C.c_int64, _P, _P, _P, _P, C.c_double, _P, C.c_uint64, C.c_int,
                        C.c_uint64, C.POINTER(_P)], C.c_int),
    "pg_pset_add": ([_P, C.c_int64, _P, _P, _P, _P, C.c_double, _P, C.c_uint64], C.c_int),
    "pg_pset_size": ([_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)], C.c_int),
    "pg_pset_get": ([_P, _P, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "pg_pset_set_tune": ([_P, C.POINTER(Tune)], C.c_int),
    "pg_execute": ([_P, _P, C.c_double, C.c_double, C.c_double, OUTPUT_CB, _P, _P,
                    C.POINTER(C.c_int64)], C.c_int),
    "pg_execute_records": ([_P, _P, C.c_double, C.c_double, C.c_double, C.c_int, RECORD_CB, _P,
                            _P, C.POINTER(C.c_int64)], C.c_int),
    "pg_pset_resort": ([_P, _P], C.c_int),
    "pg_pset_moments": ([_P, C.POINTER(C.c_double), _P], C.c_int),
    "pg_pset_save": ([_P, C.c_char_p], C.c_int),
    "pg_pset_restore": ([_P, C.c_char_p, C.POINTER(_P)], C.c_int),
    "pg_pset_destroy": ([_P], C.c_int),
    "pg_debug_set_alloc_limit": ([C.c_int64], C.c_int),
    "pg_debug_bounded_wait": ([C.c_int64, C.c_void_p], C.c_int),
    "pg_pset_kernel_timing": ([_P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int64)], C.c_int),
    "pg_launch_count": ([C.POINTER(C.c_int64)], C.c_int),
    "pg_measure_l2_read": ([C.c_size_t, C.c_int, C.POINTER(C.c_double), _P], C.c_int),
    "pg_fieldset_stats": ([_P, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64)], C.c_int),
    "pg_moments_f64_noalloc": ([_P, _P, _P, _P, C.c_int64, _P, _P], C.c_int),
    "pg_execute_batch": ([C.c_int, _P, _P, _P, _P, C.c_double, C.POINTER(Tune), C.POINTER(Tune),
                          C.c_char_p, C.c_int, _P, C.POINTER(C.c_int64)], C.c_int),
    "pg_surrogate_features": ([_P, _P, _P], C.c_int),
    "pg_surrogate_apply": ([_P, _P, C.c_double, _P], C.c_int),
    "pg_pset_displacement": ([_P, _P, _P, _P], C.c_int),
    "pg_surrogate_run": ([_P, _P, _P, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                          C.POINTER(SurrogateStats), _P], C.c_int),
    "pg_mlp_create": ([C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64, C.POINTER(_P)], C.c_int),
    "pg_mlp_destroy": ([_P], C.c_int),
    "pg_mlp_num_params": ([_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)], C.c_int),
    "pg_mlp_get_params": ([_P, _P], C.c_int),
    "pg_mlp_set_params": ([_P, _P], C.c_int),
    "pg_mlp_set_engine": ([_P, C.c_int], C.c_int),
    "pg_mlp_forward": ([_P, _P, C.c_int64, _P, _P], C.c_int),
    "pg_mlp_grad": ([_P, _P, _P, C.c_int64, C.POINTER(C.c_float), _P, _P], C.c_int),
    "pg_mlp_train_step": ([_P, _P, _P, C.c_int64, C.c_float, C.POINTER(C.c_float), _P], C.c_int),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the shared library (building it first if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path) or os.environ.get("PG_BUILD_DIR"):
            if not build_if_missing:
                raise ImportError(f"CUDA library not built: {path}")
            _build.build()
        lib = C.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def exported_names():
    return list(_SIGS)


def check(code: int):
    if code != PG_OK:
        msg = load().pg_last_error().decode(errors="replace")
        raise PGError(code, msg)
    return code
