"""Shared helpers of the parity tests: run the oracle and the CUDA library on the
same seeded inputs and compare them."""
from __future__ import annotations

import os

import numpy as np

import oracle as O

DAY = 86400.0
BEH = {"brownian": O.BROWNIAN, "sink": O.SINK}


def oracle_field(spec, data=None):
    d = spec.data if data is None else data
    return O.Field(spec.lon, spec.lat, spec.depth, spec.times, d, spec.mesh, spec.periodic_lon,
                   spec.period)


def oracle_run(field, lon, lat, depth, t0, dt, runtime, output_dt=0.0, scheme="rk4",
               behaviours=(), kh=0.0, w_sink=0.0, seed=0, ids=None, time=None):
    """Run the oracle; returns {output time: state dict} with the final state
    under the key 'final'."""
    n = len(lon)
    st = dict(lon=np.array(lon, dtype=np.float64), lat=np.array(lat, dtype=np.float64),
              depth=np.zeros(n) if depth is None else np.array(depth, dtype=np.float64),
              time=np.full(n, t0, dtype=np.float64) if time is None else np.array(time, np.float64),
              ids=np.arange(n, dtype=np.uint64) if ids is None else np.asarray(ids, np.uint64),
              step=np.zeros(n, dtype=np.uint32), status=np.zeros(n, dtype=np.uint8))
    bits = 0
    for b in behaviours:
        bits |= BEH[b]
    k = O.Kernel(O.RK4 if scheme == "rk4" else O.EULER, bits, kh, w_sink, seed)
    sgn = 1.0 if dt > 0 else -1.0
    t_begin = st["time"].min() if dt > 0 else st["time"].max()
    t_end = t_begin + sgn * runtime
    outs = {}
    stops = []
    if output_dt > 0:
        m = 1
        while sgn * (t_end - (t_begin + sgn * m * output_dt)) > 0:
            stops.append(t_begin + sgn * m * output_dt)
            m += 1
    stops.append(t_end)
    steps = 0
    for ts in stops:
        steps += O.run(field, k, st["lon"], st["lat"], st["depth"], st["time"], st["ids"],
                       st["step"], st["status"], dt, ts, t_end)
        outs[ts] = {kk: v.copy() for kk, v in st.items()}
    outs["final"] = outs[t_end]
    outs["steps"] = steps
    return outs


def gpu_run(pset, kernel, runtime, dt, output_dt=0.0):
    outs = {}

    def hook(t, d):
        o = np.argsort(d["id"], kind="stable")
        outs[t] = {k: v[o] for k, v in d.items()}
    steps = pset.execute(kernel, runtime, dt, output_dt, hook if output_dt > 0 else None)
    outs["final"] = pset.get()
    outs["steps"] = steps
    return outs


def assert_close_positions(g, o, tol_abs, what=""):
    """Positions equal within tol_abs (per axis), deleted sets equal."""
    np.testing.assert_array_equal(g["status"], o["status"], err_msg=f"status {what}")
    for ax in ("lon", "lat", "depth"):
        np.testing.assert_allclose(g[ax], o[ax], rtol=0, atol=tol_abs[ax] if isinstance(tol_abs, dict)
                                   else tol_abs, err_msg=f"{ax} {what}")


def cell_error(g, o, spec, periodic=True):
    """Per-particle position error in cell units (uniform horizontal axes;
    depth in units of the local layer thickness)."""
    dx = (spec.lon[-1] - spec.lon[0]) / (len(spec.lon) - 1)
    dy = (spec.lat[-1] - spec.lat[0]) / (len(spec.lat) - 1)
    dlon = g["lon"] - o["lon"]
    if periodic:
        dlon = (dlon + 180.0) % 360.0 - 180.0
    e = [np.abs(dlon) / dx, np.abs(g["lat"] - o["lat"]) / dy]
    if len(spec.depth) > 1:
        k = np.clip(np.searchsorted(spec.depth, o["depth"]) - 1, 0, len(spec.depth) - 2)
        dz = spec.depth[k + 1] - spec.depth[k]
        e.append(np.abs(g["depth"] - o["depth"]) / dz)
    return np.max(np.stack(e), axis=0)


def paper_value(key):
    """A value the paper prints for one of its test cases, from
    tests/golden/paper_reported_values.txt (each line cites its section)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "paper_reported_values.txt")
    for line in open(path):
        parts = line.split()
        if parts and not parts[0].startswith("#") and parts[0] == key:
            return float(parts[1])
    raise KeyError(key)
