"""Seeded synthetic velocity fields shaped like the paper's workloads.

Every generator returns a :class:`FieldSpec`: rectilinear axes (Sect. 2.4),
snapshot times and node values of U, V[, W] laid out (nt, nfields, nz, ny, nx)
with longitude fastest.  Node values come from closed-form formulas or from a
seeded random spectrum; nothing here interpolates or integrates.

Idealised flows follow the paper's validation cases (Sect. 4.2): solid-body
rotation, uniform zonal flow on a sphere, time-oscillating zonal flow, flow
around a peninsula, a Stommel-like gyre, a translating decaying eddy (stand-in
for the damped inertial oscillation, whose formula the paper does not print)
and a zero field for Brownian motion.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Optional

import numpy as np

FLAT, SPHERICAL = 0, 1
DAY = 86400.0
EARTH_R = 6371.0e3

__all__ = [
    "FLAT", "SPHERICAL", "DAY", "FieldSpec", "GlobalField", "solid_body_rotation",
    "zonal_flow_sphere", "oscillating_flow", "peninsula", "peninsula_psi",
    "stommel_gyre", "stommel_psi", "decaying_eddy", "eddy_trajectory", "zero_field",
    "uniform_flow", "linear_field", "global_axes", "temperature", "temperature_base",
    "temperature_at",
]


@dataclasses.dataclass
class FieldSpec:
    lon: np.ndarray
    lat: np.ndarray
    depth: np.ndarray
    times: np.ndarray
    data: Optional[np.ndarray]          # (nt, nf, nz, ny, nx) or None when generated per slab
    mesh: int = FLAT
    periodic_lon: bool = False
    period: float = 0.0
    nfields: int = 2
    slab: Optional[Callable[[int], np.ndarray]] = None   # s -> (nf, nz, ny, nx)

    @property
    def nt(self):
        return len(self.times)

    def snapshot(self, s):
        if self.data is not None:
            return self.data[s]
        return self.slab(s)


def _axes_flat(x0, x1, nx, y0, y1, ny):
    return np.linspace(x0, x1, nx), np.linspace(y0, y1, ny)


def solid_body_rotation(half_width=10e3, res=100.0, period=DAY):
    """Counter-clockwise rotation (u, v) = (-omega y, omega x), Sect. 4.2.1."""
    n = int(round(2 * half_width / res)) + 1
    x, y = _axes_flat(-half_width, half_width, n, -half_width, half_width, n)
    omega = 2 * np.pi / period
    X, Y = np.meshgrid(x, y)
    data = np.stack([-omega * Y, omega * X])[None, :, None]
    return FieldSpec(x, y, np.zeros(1), np.zeros(1), data)


def uniform_flow(u=0.3, v=-0.2, n=5, half_width=1e6):
    x, y = _axes_flat(-half_width, half_width, n, -half_width, half_width, n)
    data = np.empty((1, 2, 1, n, n))
    data[0, 0] = u
    data[0, 1] = v
    return FieldSpec(x, y, np.zeros(1), np.zeros(1), data)


def zonal_flow_sphere(u=1.0, res=1.0):
    """Uniform 1 m/s eastward flow on a global periodic 1-degree grid, Sect. 4.2.2."""
    lon = np.arange(0.0, 360.0, res)
    lat = np.arange(-90.0 + res / 2, 90.0, res)
    data = np.zeros((1, 2, 1, len(lat), len(lon)))
    data[0, 0] = u
    return FieldSpec(lon, lat, np.zeros(1), np.zeros(1), data, SPHERICAL, True)


def oscillating_flow(A=0.1, period=DAY, dt_snap=300.0, days=4.0, half_width=1e5):
    """u = A cos(omega t), v = A, uniform in space, snapshots every 5 min, Sect. 4.2.3."""
    nt = int(round(days * DAY / dt_snap)) + 1
    times = np.arange(nt) * dt_snap
    x, y = _axes_flat(-half_width, half_width, 3, -half_width, half_width, 3)
    data = np.empty((nt, 2, 1, 3, 3))
    data[:, 0] = (A * np.cos(2 * np.pi / period * times))[:, None, None, None]
    data[:, 1] = A
    return FieldSpec(x, y, np.zeros(1), times, data)


def peninsula_psi(x, y, U=1.0, R=22224.0, xc=55560.0):
    r2 = (x - xc) ** 2 + y ** 2
    return -U * y * (1.0 - R * R / r2)


def peninsula(nx=101, ny=51, Lx=111120.0, Ly=55560.0, U=1.0, R=22224.0):
    """Potential flow past a half-cylinder on the southern edge (Sect. 4.2.4).

    The paper cites the streamfunction without printing it; this is the
    textbook one, psi = -U y (1 - R^2/r^2), u = -dpsi/dy, v = dpsi/dx,
    with zero velocity on land (r < R).  Flat mesh in metres on a
    1 deg x 0.5 deg box (1 deg = 111.12 km) at 1/100 deg.
    """
    xc = Lx / 2
    x, y = _axes_flat(0.0, Lx, nx, 0.0, Ly, ny)
    X, Y = np.meshgrid(x, y)
    r2 = (X - xc) ** 2 + Y ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        u = U * (1.0 - R * R / r2 + 2.0 * R * R * Y * Y / r2 ** 2)
        v = -2.0 * U * R * R * Y * (X - xc) / r2 ** 2
    land = r2 < R * R
    u[land] = 0.0
    v[land] = 0.0
    data = np.stack([u, v])[None, :, None]
    return FieldSpec(x, y, np.zeros(1), np.zeros(1), data)


def stommel_psi(x, y, L=1e6, psi0=1e5):
    return psi0 * np.sin(np.pi * y / L) * (1.0 - x / L - np.exp(-x / (L / 20.0)))


def stommel_gyre(n=201, L=1e6, psi0=1e5):
    """Steady Stommel-like gyre with a western boundary current.

    psi = Psi0 sin(pi y/L) (1 - x/L - exp(-x/(L/20))); u = -dpsi/dy and
    v = dpsi/dx are evaluated analytically at the nodes.  FP64, flat mesh.
    """
    x, y = _axes_flat(0.0, L, n, 0.0, L, n)
    X, Y = np.meshgrid(x, y)
    g = 1.0 - X / L - np.exp(-X / (L / 20.0))
    dg = -1.0 / L + (20.0 / L) * np.exp(-X / (L / 20.0))
    u = -psi0 * (np.pi / L) * np.cos(np.pi * Y / L) * g
    v = psi0 * np.sin(np.pi * Y / L) * dg
    data = np.stack([u, v])[None, :, None]
    return FieldSpec(x, y, np.zeros(1), np.zeros(1), data)


def decaying_eddy(c=(0.05, 0.02), omega0=2 * np.pi / DAY, tau=2 * DAY, dt_snap=300.0,
                  days=4.0, half_width=2e4, n=41):
    """Translating decaying eddy: v(x,t) = c + omega0 e^{-t/tau} k x (x - c t).

    Linear in space, so bilinear interpolation is exact; the closed-form path
    is given by :func:`eddy_trajectory`.
    """
    nt = int(round(days * DAY / dt_snap)) + 1
    times = np.arange(nt) * dt_snap
    lo = -half_width
    hi = half_width + max(c) * days * DAY
    x, y = _axes_flat(lo, hi, n, lo, hi, n)
    X, Y = np.meshgrid(x, y)
    data = np.empty((nt, 2, 1, n, n))
    for s, t in enumerate(times):
        w = omega0 * np.exp(-t / tau)
        data[s, 0, 0] = c[0] - w * (Y - c[1] * t)
        data[s, 1, 0] = c[1] + w * (X - c[0] * t)
    return FieldSpec(x, y, np.zeros(1), times, data)


def eddy_trajectory(x0, y0, t, c=(0.05, 0.02), omega0=2 * np.pi / DAY, tau=2 * DAY):
    r = np.hypot(x0, y0)
    th0 = np.arctan2(y0, x0)
    th = th0 + omega0 * tau * (1.0 - np.exp(-t / tau))
    return c[0] * t + r * np.cos(th), c[1] * t + r * np.sin(th)


def zero_field(half_width=30e3, n=61):
    x, y = _axes_flat(-half_width, half_width, n, -half_width, half_width, n)
    return FieldSpec(x, y, np.zeros(1), np.zeros(1), np.zeros((1, 2, 1, n, n)))


def linear_field(rng, nx=7, ny=6, nz=5, nt=3, nfields=3, mesh=FLAT, stretched=True):
    """f = a + b x + c y + d z + e t on random (optionally stretched) axes.

    Bi/trilinear and linear-in-time interpolation reproduce such a field
    exactly, which pins the interpolation weights.
    """
    def axis(n, lo, hi):
        if n == 1:
            return np.array([lo])
        if stretched:
            d = rng.uniform(0.5, 1.5, n - 1)
            return lo + (hi - lo) * np.concatenate([[0.0], np.cumsum(d)]) / d.sum()
        return np.linspace(lo, hi, n)
    if mesh == SPHERICAL:
        lon, lat = axis(nx, 10.0, 30.0), axis(ny, -40.0, -20.0)
    else:
        lon, lat = axis(nx, -5e3, 7e3), axis(ny, 1e3, 9e3)
    depth = axis(nz, 5.0, 500.0) if nz > 1 else np.zeros(1)
    times = axis(nt, 0.0, 3 * DAY) if nt > 1 else np.zeros(1)
    coef = rng.normal(size=(nfields, 5))
    T, Z, Y, X = np.meshgrid(times, depth, lat, lon, indexing="ij")
    data = np.stack([c[0] + c[1] * X * 1e-3 + c[2] * Y * 1e-3 + c[3] * Z * 1e-2
                     + c[4] * T / DAY for c in coef], axis=1)
    return FieldSpec(lon, lat, depth, times, data, mesh, False, 0.0, nfields), coef


# --------------------------------------------------------------------------
# Global random fields (configurations with 1/4 and 1/12 degree grids).
# --------------------------------------------------------------------------

def global_axes(res_deg, nz=1, z0=5.0, z1=5000.0):
    """Periodic global lon [0, 360), cell-centred lat, geometric depth z0..z1."""
    nx = int(round(360.0 / res_deg))
    ny = int(round(180.0 / res_deg))
    lon = np.arange(nx) * (360.0 / nx)
    lat = -90.0 + (180.0 / ny) * (np.arange(ny) + 0.5)
    if nz > 1:
        depth = z0 * (z1 / z0) ** (np.arange(nz) / (nz - 1))
    else:
        depth = np.zeros(1)
    return lon, lat, depth


class GlobalField:
    """Seeded random velocity on a global grid with a k^-3 energy spectrum.

    Per snapshot, a horizontal streamfunction psi is summed from random-phase
    modes with amplitude k^-3 (energy spectrum k^-3), tapered by cos^2(lat);
    u = -(1/R) dpsi/dlat, v = 1/(R cos lat) dpsi/dlon (central differences),
    scaled to a surface rms speed ``rms_uv`` and multiplied by exp(-z/1000 m).
    Each mode's phase turns an integer number of times per ``period``, so the
    field is exactly periodic.  W is an independent random field of rms
    ``rms_w`` times sin(pi (z - z0)/(z1 - z0)), which vanishes at the top and
    bottom levels.  Values are stored as float32.
    """

    def __init__(self, res_deg=0.25, nz=50, nt=30, seed=2, rms_uv=0.3, rms_w=1e-4,
                 period=30 * DAY, kmax=90, with_w=True):
        self.lon, self.lat, self.depth = global_axes(res_deg, nz)
        self.nx, self.ny, self.nz = len(self.lon), len(self.lat), len(self.depth)
        self.times = np.arange(nt) * (period / nt)
        self.period = period
        self.with_w = with_w and nz > 1
        self.nfields = 3 if self.with_w else 2
        rng = np.random.default_rng(seed)
        ky = np.fft.fftfreq(self.ny, 1.0 / self.ny)[:, None]
        kx = np.fft.rfftfreq(self.nx, 1.0 / self.nx)[None, :]
        k = np.hypot(kx, ky)
        amp = np.where((k >= 1.0) & (k <= kmax), np.maximum(k, 1.0) ** -3.0, 0.0)
        shp = amp.shape
        self._amp = amp
        self._phase = rng.uniform(0.0, 2 * np.pi, shp)
        self._freq = rng.choice(np.array([-2.0, -1.0, 1.0, 2.0]), shp)
        self._phase_w = rng.uniform(0.0, 2 * np.pi, shp)
        self._freq_w = rng.choice(np.array([-2.0, -1.0, 1.0, 2.0]), shp)
        self._taper = np.cos(np.deg2rad(self.lat))[:, None] ** 2
        self._coslat = np.cos(np.deg2rad(self.lat))[:, None]
        self.prof_uv = np.exp(-self.depth / 1000.0) if nz > 1 else np.ones(1)
        if nz > 1:
            self.prof_w = np.sin(np.pi * (self.depth - self.depth[0]) /
                                 (self.depth[-1] - self.depth[0]))
            self.prof_w[0] = 0.0
            self.prof_w[-1] = 0.0
        else:
            self.prof_w = np.zeros(1)
        u0, v0 = self._uv2d_raw(0)
        self._scale_uv = rms_uv / np.sqrt(np.mean(u0 ** 2 + v0 ** 2))
        self._scale_w = 0.0
        if self.with_w:
            w0 = self._w2d_raw(0)
            self._scale_w = rms_w / np.sqrt(np.mean(w0 ** 2))

    def _psi(self, s, phase, freq):
        t = self.times[s]
        spec = self._amp * np.exp(1j * (phase + 2 * np.pi * freq * t / self.period))
        return np.fft.irfft2(spec, s=(self.ny, self.nx)) * (self.nx * self.ny)

    def _uv2d_raw(self, s):
        psi = self._psi(s, self._phase, self._freq) * self._taper
        dlam = np.deg2rad(360.0 / self.nx)
        dphi = np.deg2rad(180.0 / self.ny)
        dpsi_dlam = (np.roll(psi, -1, axis=1) - np.roll(psi, 1, axis=1)) / (2 * dlam)
        dpsi_dphi = np.gradient(psi, dphi, axis=0)
        u = -dpsi_dphi / EARTH_R
        v = dpsi_dlam / (EARTH_R * self._coslat)
        return u, v

    def _w2d_raw(self, s):
        return self._psi(s, self._phase_w, self._freq_w) * self._taper

    def base2d(self, s):
        """Surface (u, v[, w]) in float64 before the vertical profiles."""
        u, v = self._uv2d_raw(s)
        out = [u * self._scale_uv, v * self._scale_uv]
        if self.with_w:
            out.append(self._w2d_raw(s) * self._scale_w)
        return np.stack(out)

    def profiles(self):
        """(nfields, nz) vertical profiles applied to the base fields."""
        rows = [self.prof_uv, self.prof_uv]
        if self.with_w:
            rows.append(self.prof_w)
        return np.stack(rows)

    def slab(self, s, base=None):
        """Snapshot s as float32 (nf, nz, ny, nx): float32(base * profile)."""
        if base is None:
            base = self.base2d(s)
        prof = self.profiles()
        out = np.empty((self.nfields, self.nz, self.ny, self.nx), dtype=np.float32)
        for f in range(self.nfields):
            for k in range(self.nz):
                out[f, k] = base[f] * prof[f, k]
        return out

    def spec(self, materialise=False):
        data = None
        if materialise:
            data = np.stack([self.slab(s) for s in range(len(self.times))])
        return FieldSpec(self.lon, self.lat, self.depth, self.times, data, SPHERICAL, True,
                         self.period, self.nfields, None if materialise else self.slab)


def _global_base2d_torch(self, s, device):
    """:meth:`GlobalField.base2d` evaluated with torch on `device` (FP64).

    Same formulas as the numpy version (values agree to rounding); used to
    build large fields quickly.  Whatever consumes a field built this way (the
    CUDA path and the oracle) must read the same arrays."""
    import torch
    t = float(self.times[s])
    amp = torch.as_tensor(self._amp, device=device)

    def psi(phase, freq):
        ph = torch.as_tensor(phase, device=device) + 2 * np.pi * torch.as_tensor(
            freq, device=device) * (t / self.period)
        spec = torch.polar(amp, ph)
        return torch.fft.irfft2(spec, s=(self.ny, self.nx)) * (self.nx * self.ny)

    taper = torch.as_tensor(self._taper, device=device)
    coslat = torch.as_tensor(self._coslat, device=device)
    p = psi(self._phase, self._freq) * taper
    dlam = np.deg2rad(360.0 / self.nx)
    dphi = np.deg2rad(180.0 / self.ny)
    dpsi_dlam = (torch.roll(p, -1, dims=1) - torch.roll(p, 1, dims=1)) / (2 * dlam)
    dpsi_dphi = torch.gradient(p, spacing=dphi, dim=0)[0]
    u = -dpsi_dphi / EARTH_R
    v = dpsi_dlam / (EARTH_R * coslat)
    out = [u * self._scale_uv, v * self._scale_uv]
    if self.with_w:
        out.append(psi(self._phase_w, self._freq_w) * taper * self._scale_w)
    return torch.stack(out)


GlobalField.base2d_torch = _global_base2d_torch


def temperature_base(lon, lat, depth, seed=9, noise=0.5, dtype=np.float64):
    """The time-independent part of :func:`temperature`, (nz, ny, nx)."""
    rng = np.random.default_rng(seed)
    lon = np.asarray(lon, np.float64)
    lat = np.asarray(lat, np.float64)
    depth = np.asarray(depth, np.float64)
    if np.max(np.abs(lat)) > 90.0:
        latd = -60.0 + 120.0 * (lat - lat.min()) / max(lat.max() - lat.min(), 1.0)
    else:
        latd = lat
    base = (2.0 + 26.0 * np.cos(np.deg2rad(latd))[None, :, None] ** 2 *
            np.exp(-depth / 700.0)[:, None, None]).astype(dtype)
    out = np.empty((len(depth), len(latd), len(lon)), dtype)
    out[...] = base
    out += (rng.standard_normal(size=out.shape, dtype=np.float32 if dtype == np.float32
                                else np.float64) * noise).astype(dtype)
    return out


def temperature_at(base, t, period=30 * DAY):
    """Snapshot of :func:`temperature` at time t from its base."""
    return base + base.dtype.type(np.sin(2 * np.pi * t / period))


def temperature(lon, lat, depth, times, seed=9, period=30 * DAY, noise=0.5):
    """Seeded synthetic sea temperature (deg C) on a grid, (nt, nz, ny, nx).

    A warm surface that cools towards the poles and with depth, 2 + 26
    cos^2(lat) exp(-z / 700 m), plus a seasonal-like swing of 1 degree with
    the given period and seeded random perturbations of rms `noise` (a
    stand-in for the OGCM temperature the worked example samples).  Flat
    grids use lat in metres scaled to +-60 degrees.
    """
    rng = np.random.default_rng(seed)
    lon = np.asarray(lon, np.float64)
    lat = np.asarray(lat, np.float64)
    depth = np.asarray(depth, np.float64)
    times = np.atleast_1d(np.asarray(times, np.float64))
    if np.max(np.abs(lat)) > 90.0:
        latd = -60.0 + 120.0 * (lat - lat.min()) / max(lat.max() - lat.min(), 1.0)
    else:
        latd = lat
    base = 2.0 + 26.0 * np.cos(np.deg2rad(latd))[None, :, None] ** 2 * \
        np.exp(-depth / 700.0)[:, None, None]
    pert = rng.normal(size=(len(depth), len(latd), len(lon))) * noise
    out = np.empty((len(times), len(depth), len(latd), len(lon)))
    for s, t in enumerate(times):
        out[s] = base + np.sin(2 * np.pi * t / period) + pert
    return out
