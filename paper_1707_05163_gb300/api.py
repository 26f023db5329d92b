"""Python binding of the C ABI (argument marshalling only; all work runs in the
CUDA library).

Mirrors the paper's objects (Lange & van Sebille, "Parcels v0.9", Sect. 2.1,
2.2, 2.4, 3): :class:`FieldSet`, :class:`ParticleSet`, :class:`Kernel` and
``ParticleSet.execute(kernel, runtime, dt, output_dt)``.  Arrays may be numpy
arrays (host) or torch tensors (host or CUDA); they are passed to the library
as raw pointers.
"""
from __future__ import annotations

import ctypes as C
from typing import Callable, Optional

import numpy as np

from . import _native as N

_MESH = {"flat": N.PG_FLAT, "spherical": N.PG_SPHERICAL}
_STORAGE = {"f64": N.PG_F64, "f32": N.PG_F32, "f16": N.PG_F16S, "bf16": N.PG_BF16S}
_POS = {"f64": N.PG_POS_F64, "f32": N.PG_POS_F32, "cell": N.PG_POS_CELL}
_INTERP = {"linear": N.PG_LINEAR, "nearest": N.PG_NEAREST}
_BEH = {"brownian": N.PG_BROWNIAN, "sink": N.PG_SINK, "settle": N.PG_SETTLE, "age": N.PG_AGE,
        "sample": N.PG_SAMPLE}


def _ptr(a, dtype):
    """(pointer, keep-alive) of a contiguous array with the element type `dtype`.

    numpy inputs are converted to `dtype`; torch tensors (host or CUDA) are
    passed as they are when their element size matches, else converted."""
    if a is None:
        return None, None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            want = {np.float64: torch.float64, np.float32: torch.float32,
                    np.uint64: torch.int64, np.uint32: torch.int32, np.uint8: torch.uint8}[dtype]
            same_int = (dtype in (np.uint64, np.uint32, np.uint8) and not a.is_floating_point()
                        and a.element_size() == np.dtype(dtype).itemsize)
            if a.dtype != want and not same_int:
                a = a.to(want)
            a = a.contiguous()
            return a.data_ptr(), a
    except ImportError:
        pass
    a = np.ascontiguousarray(a, dtype=dtype)
    return a.ctypes.data, a


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return getattr(stream, "cuda_stream", stream)


def _src_dtype(a):
    try:
        import torch
        if isinstance(a, torch.Tensor):
            return N.PG_F64 if a.dtype == torch.float64 else N.PG_F32
    except ImportError:
        pass
    return N.PG_F64 if np.asarray(a).dtype == np.float64 else N.PG_F32


class FieldSet:
    """Rectilinear U, V[, W] velocity fields (Sect. 2.4)."""

    def __init__(self, lon, lat, depth=None, mesh="flat", periodic_lon=False, nfields=2,
                 storage="f32"):
        self._lib = N.load()
        lon = np.ascontiguousarray(lon, dtype=np.float64)
        lat = np.ascontiguousarray(lat, dtype=np.float64)
        depth = np.ascontiguousarray(np.zeros(1) if depth is None else depth, dtype=np.float64)
        self.lon, self.lat, self.depth = lon, lat, depth
        self.nfields = nfields
        self.storage = storage
        g = N.Grid(len(lon), len(lat), len(depth), lon.ctypes.data, lat.ctypes.data,
                   depth.ctypes.data)
        h = C.c_void_p()
        N.check(self._lib.pg_fieldset_create(C.byref(g), _MESH[mesh], int(bool(periodic_lon)),
                                             nfields, _STORAGE[storage], C.byref(h)))
        self.h = h
        self._keep = []
        self._cb = None

    @property
    def shape(self):
        return (self.nfields, len(self.depth), len(self.lat), len(self.lon))

    def set_times(self, times, period=0.0):
        t = np.ascontiguousarray(np.atleast_1d(times), dtype=np.float64)
        N.check(self._lib.pg_fieldset_set_times(self.h, len(t), t.ctypes.data, float(period)))
        self.times = t

    def load_snapshot(self, s, data, stream=None):
        """Snapshot s, shaped (nfields, nz, ny, nx), float32/float64, host or device."""
        dt = _src_dtype(data)
        p, keep = _ptr(data, np.float64 if dt == N.PG_F64 else np.float32)
        N.check(self._lib.pg_fieldset_load_snapshot(self.h, int(s), p, dt, _stream(stream)))

    def set_ring(self, slots):
        """Slots of the streamed-snapshot ring (4..64), before :meth:`stream`."""
        N.check(self._lib.pg_fieldset_set_ring(self.h, int(slots)))

    def stream(self, snapshots=None, callback: Optional[Callable] = None, dtype="f32"):
        """Stream snapshots during execute: either a list of per-snapshot arrays
        (kept alive by this object) or ``callback(s, out)`` filling a numpy view
        of the pinned staging buffer."""
        if snapshots is not None:
            ptrs = []
            self._keep = []
            for a in snapshots:
                p, keep = _ptr(a, np.float64 if dtype == "f64" else np.float32)
                ptrs.append(p)
                self._keep.append(keep)
            arr = (C.c_void_p * len(ptrs))(*ptrs)
            self._keep.append(arr)
            N.check(self._lib.pg_fieldset_stream(self.h, arr, N.SNAPSHOT_CB(), None,
                                                 _STORAGE[dtype]))
        else:
            npdt = np.float64 if dtype == "f64" else np.float32
            shape = self.shape

            def cb(user, s, dst, nbytes):
                try:
                    out = np.ctypeslib.as_array((C.c_char * nbytes).from_address(dst))
                    out = out.view(npdt).reshape(shape)
                    r = callback(s, out)
                    return 0 if r is None else int(r)
                except Exception:  # a failing source aborts the execute
                    return 1
            self._cb = N.SNAPSHOT_CB(cb)
            N.check(self._lib.pg_fieldset_stream(self.h, None, self._cb, None, _STORAGE[dtype]))

    def add_constant(self, name, value):
        """A named constant read by the behaviours (Sect. 3): "Kh", "w_sink",
        "dwelling_depth", "max_age"."""
        N.check(self._lib.pg_fieldset_add_constant(self.h, name.encode(), float(value)))

    def get_constant(self, name):
        v = C.c_double()
        N.check(self._lib.pg_fieldset_get_constant(self.h, name.encode(), C.byref(v)))
        return v.value

    def set_interp(self, method):
        """Spatial interpolation of the velocities: "linear" or "nearest"."""
        N.check(self._lib.pg_fieldset_set_interp(self.h, _INTERP[method]))

    def add_scalar(self, name, method="linear"):
        """A scalar field (e.g. temperature) to sample into particle variables;
        returns its index."""
        i = C.c_int()
        N.check(self._lib.pg_fieldset_add_scalar(self.h, name.encode(), _INTERP[method],
                                                 C.byref(i)))
        self.nscalars = i.value + 1
        return i.value

    def load_scalar(self, index, s, data, stream=None):
        """Snapshot s of scalar field `index`, shaped (nz, ny, nx)."""
        dt = _src_dtype(data)
        p, keep = _ptr(data, np.float64 if dt == N.PG_F64 else np.float32)
        N.check(self._lib.pg_fieldset_load_scalar(self.h, int(index), int(s), p, dt,
                                                  _stream(stream)))

    def device_bytes(self):
        b = C.c_size_t()
        N.check(self._lib.pg_fieldset_device_bytes(self.h, C.byref(b)))
        return b.value

    def scale(self, s, f):
        v = C.c_float()
        N.check(self._lib.pg_fieldset_get_scale(self.h, s, f, C.byref(v)))
        return np.float32(v.value)

    def destroy(self):
        if self.h:
            self._lib.pg_fieldset_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    @classmethod
    def from_spec(cls, spec, storage="f32", stream=None, snapshots="resident"):
        """Build from a synthetic :class:`synth.FieldSpec` (all snapshots resident)."""
        fs = cls(spec.lon, spec.lat, spec.depth if len(spec.depth) > 1 else None,
                 mesh="spherical" if spec.mesh == 1 else "flat", periodic_lon=spec.periodic_lon,
                 nfields=spec.nfields if spec.data is None else spec.data.shape[1],
                 storage=storage)
        fs.set_times(spec.times, spec.period)
        for s in range(len(spec.times)):
            fs.load_snapshot(s, spec.snapshot(s), stream)
        return fs


class Kernel:
    """Advection scheme plus behaviours (Sect. 2.1.2): ``Kernel('rk4') + 'brownian'``.

    Behaviours: "brownian", "sink", "settle", "age", "sample".  kh / w_sink
    None: the field set's constants "Kh" / "w_sink" at execute time."""

    def __init__(self, scheme="rk4", behaviours=(), kh=0.0, w_sink=0.0):
        self._lib = N.load()
        self.scheme = scheme
        self.behaviours = tuple(behaviours)
        self.kh = float("nan") if kh is None else float(kh)
        self.w_sink = float("nan") if w_sink is None else float(w_sink)
        bits = 0
        for b in self.behaviours:
            bits |= _BEH[b]
        h = C.c_void_p()
        N.check(self._lib.pg_kernel_create({"euler": N.PG_EULER, "rk4": N.PG_RK4,
                                            "rkf45": N.PG_RKF45}[scheme], bits,
                                           self.kh, self.w_sink, C.byref(h)))
        self.h = h

    def __add__(self, other):
        if isinstance(other, str):
            other = (other,)
        return Kernel(self.scheme, self.behaviours + tuple(other), self.kh, self.w_sink)

    def __del__(self):
        try:
            if self.h:
                self._lib.pg_kernel_destroy(self.h)
                self.h = None
        except Exception:
            pass


class ParticleSet:
    """Particles on a field set (Sect. 2.1); positions kept on the device."""

    def __init__(self, fieldset: FieldSet, lon, lat, depth=None, time=None, t0=0.0, ids=None,
                 id_base=0, pos="f32", seed=0, _handle=None):
        self._lib = N.load()
        self.fieldset = fieldset
        self.pos = pos
        if _handle is not None:
            self.h = _handle
            self.fieldset_nvar = getattr(fieldset, "nscalars", 0)
            return
        n = len(lon)
        pl, k1 = _ptr(lon, np.float64)
        pa, k2 = _ptr(lat, np.float64)
        pd, k3 = _ptr(depth, np.float64)
        pt, k4 = _ptr(time, np.float64)
        pi, k5 = _ptr(ids, np.uint64)
        h = C.c_void_p()
        N.check(self._lib.pg_pset_create(fieldset.h, n, pl, pa, pd, pt, float(t0), pi,
                                         int(id_base), _POS[pos], int(seed), C.byref(h)))
        self.h = h
        self.fieldset_nvar = getattr(fieldset, "nscalars", 0)

    def add(self, lon, lat, depth=None, time=None, t0=0.0, ids=None, id_base=0):
        pl, k1 = _ptr(lon, np.float64)
        pa, k2 = _ptr(lat, np.float64)
        pd, k3 = _ptr(depth, np.float64)
        pt, k4 = _ptr(time, np.float64)
        pi, k5 = _ptr(ids, np.uint64)
        N.check(self._lib.pg_pset_add(self.h, len(lon), pl, pa, pd, pt, float(t0), pi,
                                      int(id_base)))

    def __len__(self):
        n = C.c_int64()
        N.check(self._lib.pg_pset_size(self.h, C.byref(n), None))
        return n.value

    def n_alive(self):
        n, a = C.c_int64(), C.c_int64()
        N.check(self._lib.pg_pset_size(self.h, C.byref(n), C.byref(a)))
        return a.value

    def set_tune(self, block=0, resort_steps=0, chunk_steps=0):
        t = N.Tune(int(block), int(resort_steps), int(chunk_steps))
        N.check(self._lib.pg_pset_set_tune(self.h, C.byref(t)))

    def execute(self, kernel: Kernel, runtime, dt, output_dt=0.0,
                output: Optional[Callable] = None, stream=None):
        """Advance by ``runtime`` seconds with steps of ``dt``; returns particle-steps.

        ``output(time, dict)`` is called every ``output_dt`` with host arrays."""
        cb = N.OUTPUT_CB()
        if output is not None:
            def hook(user, t, n, ids, lon, lat, dep, st):
                try:
                    def arr(p, ct, dt):
                        return np.ctypeslib.as_array((ct * n).from_address(p)).view(dt).copy() \
                            if n else np.zeros(0, dt)
                    output(t, dict(id=arr(ids, C.c_uint64, np.uint64),
                                   lon=arr(lon, C.c_double, np.float64),
                                   lat=arr(lat, C.c_double, np.float64),
                                   depth=arr(dep, C.c_double, np.float64),
                                   status=arr(st, C.c_uint8, np.uint8)))
                    return 0
                except Exception:
                    return 1
            cb = N.OUTPUT_CB(hook)
        steps = C.c_int64()
        N.check(self._lib.pg_execute(self.h, kernel.h, float(runtime), float(dt), float(output_dt),
                                     cb, None, _stream(stream), C.byref(steps)))
        return steps.value

    def execute_records(self, kernel: Kernel, runtime, dt, output_dt, record: Callable,
                        indexed=True, stream=None):
        """Advance like :meth:`execute`, with the ParticleFile output of Sect. 3:
        ``record(time, dict)`` gets, at every output time, host copies of the
        rows (id, lon, lat, depth, status, age, vars [nvar, rows]): every
        particle, or (indexed) those alive at that time and those deleted
        since the previous output.  Returns particle-steps."""
        def hook(user, rp):
            try:
                r = rp.contents
                n = r.n

                def arr(p, ct, dt, m=n):
                    return np.ctypeslib.as_array((ct * m).from_address(p)).view(dt).copy() \
                        if m else np.zeros(0, dt)
                out = dict(id=arr(r.id, C.c_uint64, np.uint64), lon=arr(r.lon, C.c_double, np.float64),
                           lat=arr(r.lat, C.c_double, np.float64),
                           depth=arr(r.depth, C.c_double, np.float64),
                           status=arr(r.status, C.c_uint8, np.uint8),
                           age=arr(r.age, C.c_double, np.float64))
                vs = np.zeros((r.nvar, n))
                for j in range(r.nvar):
                    if n:
                        vs[j] = np.ctypeslib.as_array(
                            (C.c_double * n).from_address(r.vars + 8 * j * r.var_stride))
                out["vars"] = vs
                res = record(r.time, out)
                return 0 if res is None else int(res)
            except Exception:
                return 1
        cb = N.RECORD_CB(hook)
        steps = C.c_int64()
        N.check(self._lib.pg_execute_records(self.h, kernel.h, float(runtime), float(dt),
                                             float(output_dt), int(bool(indexed)), cb, None,
                                             _stream(stream), C.byref(steps)))
        return steps.value

    def get(self, sort_by_id=True, stream=None):
        """Host copy of the state: dict of lon, lat, depth, time, id, step, status."""
        n = len(self)
        out = dict(lon=np.empty(n), lat=np.empty(n), depth=np.empty(n), time=np.empty(n),
                   id=np.empty(n, np.uint64), step=np.empty(n, np.uint32),
                   status=np.empty(n, np.uint8))
        if n:
            N.check(self._lib.pg_pset_get(self.h, out["lon"].ctypes.data, out["lat"].ctypes.data,
                                          out["depth"].ctypes.data, out["time"].ctypes.data,
                                          out["id"].ctypes.data, out["step"].ctypes.data,
                                          out["status"].ctypes.data, _stream(stream)))
        if sort_by_id and n:
            o = np.argsort(out["id"], kind="stable")
            out = {k: v[o] for k, v in out.items()}
        return out

    def get_variables(self, sort_by_id=True, stream=None):
        """Host copy of the particle variables: dict of age [n] and vars
        [nvar, n] (sampled scalar fields), in id order by default."""
        n = len(self)
        nvar = self.fieldset_nvar
        age = np.empty(n)
        var = np.empty((nvar, n))
        if n:
            N.check(self._lib.pg_pset_get_variables(self.h, age.ctypes.data,
                                                    var.ctypes.data if nvar else None,
                                                    _stream(stream)))
            if sort_by_id:
                ids = np.empty(n, np.uint64)
                N.check(self._lib.pg_pset_get(self.h, None, None, None, None, ids.ctypes.data,
                                              None, None, _stream(stream)))
                o = np.argsort(ids, kind="stable")
                age, var = age[o], var[:, o]
        return dict(age=age, vars=var)

    def get_into(self, lon=None, lat=None, depth=None, time=None, ids=None, status=None,
                 stream=None):
        """Copy the state into caller buffers (numpy or torch, host or device)."""
        ps = [_ptr(a, d)[0] if a is not None else None for a, d in
              ((lon, np.float64), (lat, np.float64), (depth, np.float64), (time, np.float64),
               (ids, np.uint64))]
        pst = _ptr(status, np.uint8)[0] if status is not None else None
        N.check(self._lib.pg_pset_get(self.h, ps[0], ps[1], ps[2], ps[3], ps[4], None, pst,
                                      _stream(stream)))

    def resort(self, stream=None):
        N.check(self._lib.pg_pset_resort(self.h, _stream(stream)))

    def moments(self, stream=None):
        out = (C.c_double * 7)()
        N.check(self._lib.pg_pset_moments(self.h, out, _stream(stream)))
        return np.array(out[:])

    def save(self, path):
        N.check(self._lib.pg_pset_save(self.h, str(path).encode()))

    @classmethod
    def restore(cls, fieldset: FieldSet, path):
        lib = N.load()
        h = C.c_void_p()
        N.check(lib.pg_pset_restore(fieldset.h, str(path).encode(), C.byref(h)))
        return cls(fieldset, None, None, _handle=h)

    def destroy(self):
        if self.h:
            self._lib.pg_pset_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def execute_batch(psets, kernels, runtimes, dts, window=86400.0, tune=None, tune_cache=None,
                  use_graph=True, stream=None):
    """Advance many releases in one persistent launch per window (pg_execute_batch).

    ``tune`` = (block, resort_windows) or None for the autotuner.  Returns
    (particle-steps, (block, resort_windows) used)."""
    lib = N.load()
    nrel = len(psets)
    ps_arr = (C.c_void_p * nrel)(*[p.h.value for p in psets])
    k_arr = (C.c_void_p * nrel)(*[k.h.value for k in kernels])
    rt = np.ascontiguousarray(runtimes, dtype=np.float64)
    dt = np.ascontiguousarray(dts, dtype=np.float64)
    t_in = N.Tune(int(tune[0]), int(tune[1]), 0) if tune is not None else None
    chosen = N.Tune()
    steps = C.c_int64()
    N.check(lib.pg_execute_batch(nrel, ps_arr, k_arr, rt.ctypes.data, dt.ctypes.data,
                                 float(window), C.byref(t_in) if t_in is not None else None,
                                 C.byref(chosen),
                                 str(tune_cache).encode() if tune_cache else None,
                                 int(bool(use_graph)), _stream(stream), C.byref(steps)))
    return steps.value, (chosen.block, chosen.resort_steps)


class MLP:
    """The surrogate network (pg_mlp_*): BF16 tensor-core products, FP32 masters."""

    def __init__(self, n_in=37, width=256, depth=4, n_out=3, seed=0):
        self._lib = N.load()
        self.n_in, self.width, self.depth, self.n_out = n_in, width, depth, n_out
        h = C.c_void_p()
        N.check(self._lib.pg_mlp_create(n_in, width, depth, n_out, int(seed), C.byref(h)))
        self.h = h

    def num_params(self):
        p, r = C.c_int64(), C.c_int64()
        N.check(self._lib.pg_mlp_num_params(self.h, C.byref(p), C.byref(r)))
        return p.value, r.value

    def get_params(self):
        out = np.empty(self.num_params()[0], dtype=np.float32)
        N.check(self._lib.pg_mlp_get_params(self.h, out.ctypes.data))
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        assert flat.size == self.num_params()[0]
        N.check(self._lib.pg_mlp_set_params(self.h, flat.ctypes.data))

    def set_engine(self, tcgen05):
        """0/False: mma.sync; 1/True: tcgen05 (fused inference where the shape
        allows); 2: tcgen05 layer by layer."""
        N.check(self._lib.pg_mlp_set_engine(self.h, int(tcgen05)))

    def forward(self, x, out=None, stream=None):
        """x: CUDA float32 tensor [M x n_in] -> CUDA float32 tensor [M x n_out]."""
        import torch
        x = x.contiguous()
        M = x.shape[0]
        if out is None:
            out = torch.empty((M, self.n_out), dtype=torch.float32, device=x.device)
        N.check(self._lib.pg_mlp_forward(self.h, x.data_ptr(), M, out.data_ptr(), _stream(stream)))
        return out

    def grad(self, x, t, stream=None):
        loss = C.c_float()
        g = np.empty(self.num_params()[0], dtype=np.float32)
        N.check(self._lib.pg_mlp_grad(self.h, x.contiguous().data_ptr(), t.contiguous().data_ptr(),
                                      x.shape[0], C.byref(loss), g.ctypes.data, _stream(stream)))
        return loss.value, g

    def train_step(self, x, t, lr, stream=None):
        loss = C.c_float()
        N.check(self._lib.pg_mlp_train_step(self.h, x.data_ptr(), t.data_ptr(), x.shape[0],
                                            float(lr), C.byref(loss), _stream(stream)))
        return loss.value

    def __del__(self):
        try:
            if self.h:
                self._lib.pg_mlp_destroy(self.h)
                self.h = None
        except Exception:
            pass


N_FEATURES = 37


def surrogate_features(pset, out=None, stream=None):
    """Inputs of the surrogate for every particle (CUDA float32 [n x 37])."""
    import torch
    n = len(pset)
    if out is None:
        out = torch.empty((n, N_FEATURES), dtype=torch.float32, device="cuda")
    N.check(N.load().pg_surrogate_features(pset.h, out.data_ptr(), _stream(stream)))
    return out


def surrogate_apply(pset, y, horizon, stream=None):
    N.check(N.load().pg_surrogate_apply(pset.h, y.contiguous().data_ptr(), float(horizon),
                                        _stream(stream)))


def displacement(a, b, out=None, stream=None):
    """Displacement from set a to set b (cells of lon/lat, 100 m of depth)."""
    import torch
    n = len(a)
    if out is None:
        out = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    N.check(N.load().pg_pset_displacement(a.h, b.h, out.data_ptr(), _stream(stream)))
    return out


def surrogate_run(pset, net, kernel, nsteps, check_every=5, horizon=86400.0, dt_check=1800.0,
                  threshold=1e-3, stream=None):
    """Network steps with periodic RK4 checks and fallback; returns the stats dict."""
    s = N.SurrogateStats()
    N.check(N.load().pg_surrogate_run(pset.h, net.h, kernel.h, int(nsteps), int(check_every),
                                      float(horizon), float(dt_check), float(threshold),
                                      C.byref(s), _stream(stream)))
    return {k: getattr(s, k) for k, _ in N.SurrogateStats._fields_}
