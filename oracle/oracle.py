"""ctypes binding of ``parcels_oracle.c`` (test infrastructure only).

The oracle follows Eq. 1 and Sect. 2.1.1, 2.1.2, 2.3, 2.4 and 4.2 of
Lange & van Sebille, "Parcels v0.9" (arXiv 1707.05163).  The C file's header
lists every reading taken where the paper is silent.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "parcels_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libparcels_oracle.so")

ALIVE, OOB_HORIZ, OOB_DEPTH, NAN, DELETED = 0, 1, 2, 3, 4
BROWNIAN, SINK, SETTLE, AGE, SAMPLE = 1, 2, 4, 8, 16
LINEAR, NEAREST = 0, 1
EULER, RK4, RKF45 = 0, 1, 2
FLAT, SPHERICAL = 0, 1
DEG_M = 1852.0 * 60.0

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
            "-shared", "-pthread", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


class _FieldSet(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("lon", C.c_void_p), ("lat", C.c_void_p), ("depth", C.c_void_p),
        ("mesh", C.c_int), ("periodic_lon", C.c_int), ("nfields", C.c_int),
        ("nt", C.c_int), ("times", C.c_void_p), ("period", C.c_double),
        ("dtype", C.c_int), ("data", C.c_void_p), ("deg_m", C.c_double),
        ("interp", C.c_int), ("ntracers", C.c_int), ("tracer", C.c_void_p * 2),
        ("tracer_interp", C.c_int * 2),
    ]


class _Kernel(C.Structure):
    _fields_ = [
        ("scheme", C.c_int), ("behaviours", C.c_uint), ("kh", C.c_double),
        ("w_sink", C.c_double), ("seed", C.c_uint64), ("dwell_depth", C.c_double),
        ("max_age", C.c_double), ("rk45_tol", C.c_double), ("rk45_hmin", C.c_double),
        ("rk45_hmax", C.c_double),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            L.or_locate.argtypes = [C.c_void_p, C.c_int, C.c_double, ip, dp]
            L.or_locate.restype = C.c_int
            L.or_locate_lon.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_double, ip, ip, dp]
            L.or_locate_lon.restype = C.c_int
            L.or_wrap_lon.argtypes = [C.c_double, C.c_double]
            L.or_wrap_lon.restype = C.c_double
            L.or_sample.argtypes = [C.POINTER(_FieldSet), C.c_double, C.c_double, C.c_double,
                                    C.c_double, dp]
            L.or_sample.restype = C.c_int
            L.or_velocity.argtypes = L.or_sample.argtypes
            L.or_velocity.restype = C.c_int
            L.or_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
            L.or_philox4x32_10.restype = None
            L.or_normal_pair.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, dp, dp]
            L.or_normal_pair.restype = None
            L.or_run.argtypes = [C.POINTER(_FieldSet), C.POINTER(_Kernel), C.c_int64] + \
                [C.c_void_p] * 10 + [C.c_double, C.c_double, C.c_double, C.c_int]
            L.or_rkf45_trial.argtypes = [C.POINTER(_FieldSet), C.c_double, C.c_double,
                                         C.c_double, C.c_double, C.c_double, dp, dp]
            L.or_rkf45_trial.restype = C.c_int
            L.or_sample_tracer.argtypes = [C.POINTER(_FieldSet), C.c_int, C.c_double,
                                           C.c_double, C.c_double, C.c_double, dp]
            L.or_sample_tracer.restype = C.c_int
            L.or_run.restype = C.c_int64
            L.or_quantise.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_void_p]
            L.or_quantise.restype = C.c_float
            L.or_dequantise.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_float, C.c_void_p]
            L.or_dequantise.restype = None
            _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class Field:
    """A rectilinear field set: axes, snapshots and the snapshot data.

    ``data`` has shape (nt, nfields, nz, ny, nx), float64 or float32, lon
    fastest.  ``period`` > 0 makes the field repeat in time with that period.
    """

    def __init__(self, lon, lat, depth, times, data, mesh=FLAT, periodic_lon=False,
                 period=0.0, deg_m=DEG_M, interp=LINEAR, tracers=(), tracer_interp=()):
        """``tracers``: up to two scalar fields (nt, nz, ny, nx) of the data's
        dtype, sampled by the SAMPLE behaviour; ``interp`` and
        ``tracer_interp``: LINEAR or NEAREST in space (time is linear)."""
        self.lon = np.ascontiguousarray(lon, dtype=np.float64)
        self.lat = np.ascontiguousarray(lat, dtype=np.float64)
        self.depth = np.ascontiguousarray(np.atleast_1d(depth), dtype=np.float64)
        self.times = np.ascontiguousarray(np.atleast_1d(times), dtype=np.float64)
        if data.dtype not in (np.float64, np.float32):
            data = data.astype(np.float64)
        self.data = np.ascontiguousarray(data)
        nt, nf, nz, ny, nx = self.data.shape
        assert (nt, nz, ny, nx) == (len(self.times), len(self.depth), len(self.lat), len(self.lon))
        assert nf in (2, 3)
        assert len(tracers) <= 2
        self.tracers = [np.ascontiguousarray(a, dtype=self.data.dtype) for a in tracers]
        for a in self.tracers:
            assert a.shape == (nt, nz, ny, nx)
        ti = list(tracer_interp) + [LINEAR] * (len(self.tracers) - len(tracer_interp))
        self.s = _FieldSet(nx, ny, nz, _ptr(self.lon), _ptr(self.lat), _ptr(self.depth),
                           int(mesh), int(bool(periodic_lon)), nf, nt, _ptr(self.times),
                           float(period), 0 if self.data.dtype == np.float64 else 1,
                           _ptr(self.data), float(deg_m), int(interp), len(self.tracers),
                           (C.c_void_p * 2)(*([_ptr(a) for a in self.tracers] +
                                              [None] * (2 - len(self.tracers)))),
                           (C.c_int * 2)(*(ti + [0] * (2 - len(ti)))))


class Kernel:
    def __init__(self, scheme=RK4, behaviours=0, kh=0.0, w_sink=0.0, seed=0, dwell_depth=0.0,
                 max_age=0.0, rk45_tol=0.0, rk45_hmin=1.0, rk45_hmax=86400.0):
        self.k = _Kernel(int(scheme), int(behaviours), float(kh), float(w_sink), int(seed),
                         float(dwell_depth), float(max_age), float(rk45_tol), float(rk45_hmin),
                         float(rk45_hmax))


def run(field: Field, kernel: Kernel, lon, lat, depth, time, ids, step, status, dt,
        t_stop, t_end=None, nthreads=None, age=None, variables=None, hstep=None):
    """Advance particles in place (arrays: float64 x4, uint64, uint32, uint8).

    Every live particle steps while its time is before ``t_stop`` and before
    ``t_end`` (in the direction of dt); the last step is shortened to land on
    ``t_end``.  ``age`` (float64 [n]) and ``variables`` (float64 [ntracers, n])
    are updated by the AGE and SAMPLE behaviours; ``hstep`` (float64 [n]) holds
    the RKF45 step lengths (0: start from dt).  Returns the number of
    particle-steps taken.
    """
    if t_end is None:
        t_end = t_stop
    if nthreads is None:
        nthreads = len(os.sched_getaffinity(0))
    for a, dt_ in ((lon, np.float64), (lat, np.float64), (depth, np.float64),
                   (time, np.float64), (ids, np.uint64), (step, np.uint32), (status, np.uint8)):
        assert a.dtype == dt_ and a.flags.c_contiguous
    n = len(lon)
    for a, shape in ((age, (n,)), (variables, (len(field.tracers), n)), (hstep, (n,))):
        if a is not None:
            assert a.dtype == np.float64 and a.flags.c_contiguous and a.shape == shape
    r = lib().or_run(C.byref(field.s), C.byref(kernel.k), n, _ptr(lon), _ptr(lat), _ptr(depth),
                     _ptr(time), _ptr(ids), _ptr(step), _ptr(status),
                     _ptr(age) if age is not None else None,
                     _ptr(variables) if variables is not None else None,
                     _ptr(hstep) if hstep is not None else None, float(dt),
                     float(t_stop), float(t_end), int(nthreads))
    if r == -2:
        raise ValueError("the SAMPLE behaviour needs the variables array")
    if r < 0:
        raise ValueError("time span outside the field's time range")
    return int(r)


def rkf45_trial(field: Field, t, lon, lat, depth, h):
    """One RKF45 trial: (status, fourth-order position, error in metres)."""
    out = (C.c_double * 3)()
    err = C.c_double()
    r = lib().or_rkf45_trial(C.byref(field.s), float(lon), float(lat), float(depth), float(t),
                             float(h), out, C.byref(err))
    return r, np.array(out[:]), err.value


def sample_tracer(field: Field, tr, t, lon, lat, depth=0.0):
    out = C.c_double()
    r = lib().or_sample_tracer(C.byref(field.s), int(tr), t, lon, lat, depth, C.byref(out))
    return r, out.value


def sample(field: Field, t, lon, lat, depth=0.0):
    out = (C.c_double * 3)()
    r = lib().or_sample(C.byref(field.s), t, lon, lat, depth, out)
    return r, np.array(out[:field.data.shape[1]])


def velocity(field: Field, t, lon, lat, depth=0.0):
    out = (C.c_double * 3)()
    r = lib().or_velocity(C.byref(field.s), t, lon, lat, depth, out)
    return r, np.array(out[:3])


def locate(x, p):
    x = np.ascontiguousarray(x, dtype=np.float64)
    i, xi = C.c_int(), C.c_double()
    r = lib().or_locate(_ptr(x), len(x), float(p), C.byref(i), C.byref(xi))
    return r, i.value, xi.value


def locate_lon(x, p, periodic=True):
    x = np.ascontiguousarray(x, dtype=np.float64)
    i0, i1, xi = C.c_int(), C.c_int(), C.c_double()
    r = lib().or_locate_lon(_ptr(x), len(x), int(periodic), float(p), C.byref(i0),
                            C.byref(i1), C.byref(xi))
    return r, i0.value, i1.value, xi.value


def wrap_lon(p, x0):
    return lib().or_wrap_lon(float(p), float(x0))


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def normal_pair(seed, pid, step):
    a, b = C.c_double(), C.c_double()
    lib().or_normal_pair(int(seed), int(pid), int(step), C.byref(a), C.byref(b))
    return a.value, b.value


def quantise(v, kind):
    """kind 0: binary16, 1: bfloat16.  Returns (uint16 codes, float32 scale)."""
    v = np.ascontiguousarray(v, dtype=np.float32)
    q = np.empty(v.shape, dtype=np.uint16)
    s = lib().or_quantise(_ptr(v), v.size, int(kind), _ptr(q))
    return q, np.float32(s)


def dequantise(q, kind, scale):
    q = np.ascontiguousarray(q, dtype=np.uint16)
    out = np.empty(q.shape, dtype=np.float64)
    lib().or_dequantise(_ptr(q), q.size, int(kind), float(scale), _ptr(out))
    return out
