"""Seeded particle start positions."""
from __future__ import annotations

import numpy as np

__all__ = ["uniform_particles", "Release", "batch_releases", "DT_DIVISORS"]


def uniform_particles(n, seed, lon_range, lat_range, depth_range=None, dtype=np.float64):
    """n particles uniform in a lon/lat(/depth) box.

    With ``dtype=np.float32`` the positions are rounded to float32 first, so a
    float32 run and the FP64 oracle start from the same values.
    """
    rng = np.random.default_rng(seed)
    lon = rng.uniform(lon_range[0], lon_range[1], n)
    lat = rng.uniform(lat_range[0], lat_range[1], n)
    if depth_range is None:
        depth = np.zeros(n)
    else:
        depth = rng.uniform(depth_range[0], depth_range[1], n)
    out = []
    for a in (lon, lat, depth):
        out.append(a.astype(dtype).astype(np.float64))
    return out[0], out[1], out[2]


# Divisors of one day between 10 min and 2 h: every release's dt is one of
# these, so its steps land on the daily snapshot times.
DT_DIVISORS = np.array([600, 720, 900, 1200, 1440, 1800, 2400, 2880, 3600, 4320, 5400, 7200],
                       dtype=np.float64)


class Release:
    """One particle release of the batched workload."""

    def __init__(self, n, dt, runtime, kind, kh=0.0, w_sink=0.0, seed=0):
        self.n, self.dt, self.runtime, self.kind = int(n), float(dt), float(runtime), int(kind)
        self.kh, self.w_sink, self.seed = float(kh), float(w_sink), int(seed)

    @property
    def steps(self):
        return int(round(self.runtime / self.dt))

    def __repr__(self):
        return (f"Release(n={self.n}, dt={self.dt}, runtime={self.runtime}, kind={self.kind}, "
                f"kh={self.kh:.3g}, w_sink={self.w_sink:.3g})")


def batch_releases(count=256, seed=4, n_min=1e3, n_max=2e6, dt_min=600.0, dt_max=7200.0,
                   days_min=5.0, days_max=90.0, scale=1.0):
    """Releases with log-uniform sizes and dt (snapped to a divisor of a day),
    uniform runtime in days (a whole number of dt) and a kernel mix drawn
    uniformly from {RK4, RK4 + Brownian, RK4 + sinking}.  Brownian K_h is
    log-uniform in [1, 100] m^2/s; sinking speed log-uniform in [1, 100] m/day.
    ``scale`` shrinks every size (for small test cases)."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_min), np.log(n_max))) * scale))
        dt_raw = np.exp(rng.uniform(np.log(dt_min), np.log(dt_max)))
        dt = DT_DIVISORS[np.argmin(np.abs(np.log(DT_DIVISORS / dt_raw)))]
        days = rng.uniform(days_min, days_max)
        runtime = max(1, int(round(days * 86400.0 / dt))) * dt
        kind = int(rng.integers(0, 3))
        kh = float(np.exp(rng.uniform(0.0, np.log(100.0)))) if kind == 1 else 0.0
        w = float(np.exp(rng.uniform(0.0, np.log(100.0)))) / 86400.0 if kind == 2 else 0.0
        out.append(Release(max(n, 1), dt, runtime, kind, kh, w, seed * 100003 + r))
    return out
