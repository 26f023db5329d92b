"""Pins of the oracle's worked-example parts (Sect. 3: sampled temperature,
age with a maximum, the sinking phase of a backward run; Sect. 2.3:
nearest-neighbour interpolation) against library routines and closed forms.
"""
import numpy as np
import pytest

import oracle as O

DAY = 86400.0


def _axes(rng, n, lo, hi, stretched):
    if stretched:
        x = np.sort(rng.uniform(lo, hi, n - 2))
        return np.concatenate([[lo], x, [hi]])
    return np.linspace(lo, hi, n)


def _state(n, lon, lat, dep, t0=0.0):
    return dict(lon=np.array(lon, np.float64), lat=np.array(lat, np.float64),
                depth=np.array(dep, np.float64), time=np.full(n, t0, np.float64),
                ids=np.arange(n, dtype=np.uint64), step=np.zeros(n, np.uint32),
                status=np.zeros(n, np.uint8))


def _run(f, k, st, dt, t_end, age=None, var=None):
    return O.run(f, k, st["lon"], st["lat"], st["depth"], st["time"], st["ids"], st["step"],
                 st["status"], dt, t_end, t_end, nthreads=1, age=age, variables=var)


@pytest.mark.parametrize("stretched", [False, True])
def test_nearest_matches_scipy_regular_grid_interpolator(stretched):
    """Nearest node in space, linear in time: against
    scipy.interpolate.RegularGridInterpolator(method='nearest') on each
    snapshot, at random points and at points exactly half-way between nodes
    (a tie goes to the lower node, scipy's rule)."""
    from scipy.interpolate import RegularGridInterpolator
    rng = np.random.default_rng(3)
    lon = _axes(rng, 9, 0.0, 8.0, stretched)
    lat = _axes(rng, 7, -3.0, 3.0, stretched)
    dep = _axes(rng, 5, 0.0, 40.0, stretched)
    times = np.array([0.0, 100.0])
    data = rng.normal(size=(2, 3, 5, 7, 9))
    f = O.Field(lon, lat, dep, times, data, interp=O.NEAREST)
    pts = np.stack([rng.uniform(lon[0], lon[-1], 300), rng.uniform(lat[0], lat[-1], 300),
                    rng.uniform(dep[0], dep[-1], 300)], axis=1)
    mids = np.stack([(lon[:-1] + lon[1:])[:6] / 2, (lat[:-1] + lat[1:])[:6] / 2,
                     (dep[:-1] + dep[1:])[[0, 1, 2, 3, 0, 1]] / 2], axis=1)
    pts = np.concatenate([pts, mids, np.stack([lon[[0, -1]], lat[[0, -1]], dep[[0, -1]]], 1)])
    for t in (0.0, 37.0, 100.0):
        tau = t / 100.0
        for p in pts:
            r, got = O.sample(f, t, p[0], p[1], p[2])
            assert r == 0
            for q in range(3):
                a, b = (RegularGridInterpolator((dep, lat, lon), data[s, q], method="nearest")(
                    [[p[2], p[1], p[0]]])[0] for s in (0, 1))
                assert got[q] == a + (b - a) * tau, (p, q, got[q], a, b)


def test_nearest_on_the_periodic_wrap_cell():
    """In the wrap cell (last node to the first one 360 degrees on), the
    nearest node is the last node or node 0: against scipy on an axis extended
    by the first node plus 360."""
    from scipy.interpolate import RegularGridInterpolator
    rng = np.random.default_rng(4)
    lon = np.arange(0.0, 360.0, 30.0)
    lat = np.linspace(-60.0, 60.0, 5)
    data = rng.normal(size=(1, 2, 1, 5, 12))
    f = O.Field(lon, lat, np.zeros(1), np.zeros(1), data, mesh=1, periodic_lon=True,
                interp=O.NEAREST)
    ext_lon = np.concatenate([lon, [360.0]])
    ext = np.concatenate([data[0, 0, 0], data[0, 0, 0][:, :1]], axis=1)
    ref = RegularGridInterpolator((lat, ext_lon), ext, method="nearest")
    for x in (331.0, 344.9, 345.0, 345.1, 359.99, -14.0, 705.0):
        y = 12.5
        r, got = O.sample(f, 0.0, x, y)
        assert r == 0
        assert got[0] == ref([[y, x % 360.0]])[0], x


def test_tracer_sampling_linear_and_nearest():
    """A scalar field linear in lon, lat, depth and time is sampled exactly by
    the linear scheme on stretched axes; a random field agrees with
    scipy.interpolate.RegularGridInterpolator (linear and nearest) per
    snapshot, blended linearly in time."""
    from scipy.interpolate import RegularGridInterpolator
    rng = np.random.default_rng(5)
    lon = _axes(rng, 10, 10.0, 20.0, True)
    lat = _axes(rng, 8, -5.0, 5.0, True)
    dep = _axes(rng, 6, 5.0, 500.0, True)
    times = np.array([0.0, 50.0, 200.0])
    L, A, Z = np.meshgrid(lon, lat, dep, indexing="ij")
    lin = np.stack([(1.5 + 0.3 * L - 0.7 * A + 0.01 * Z + 0.002 * t).transpose(2, 1, 0)
                    for t in times])
    rnd = rng.normal(size=(3, 6, 8, 10))
    vel = np.zeros((3, 3, 6, 8, 10))
    f = O.Field(lon, lat, dep, times, vel, tracers=(lin, rnd), tracer_interp=(O.LINEAR, O.NEAREST))
    g = O.Field(lon, lat, dep, times, vel, tracers=(rnd,), tracer_interp=(O.LINEAR,))
    for _ in range(200):
        x, y, z = rng.uniform(10, 20), rng.uniform(-5, 5), rng.uniform(5, 500)
        t = rng.uniform(0, 200)
        r, v = O.sample_tracer(f, 0, t, x, y, z)
        assert r == 0
        assert abs(v - (1.5 + 0.3 * x - 0.7 * y + 0.01 * z + 0.002 * t)) < 1e-12
        s = 0 if t < 50 else 1
        tau = (t - times[s]) / (times[s + 1] - times[s])
        for fld, tr, method in ((f, 1, "nearest"), (g, 0, "linear")):
            a, b = (RegularGridInterpolator((dep, lat, lon), rnd[q], method=method)([[z, y, x]])[0]
                    for q in (s, s + 1))
            r, v = O.sample_tracer(fld, tr, t, x, y, z)
            assert abs(v - (a + (b - a) * tau)) < 1e-12, (method, v, a, b)


def _still_3d(w=0.0, nz=31):
    """Zero horizontal velocity, uniform W (m/s), flat 3-D box 0..3000 m."""
    lon = np.linspace(0.0, 1e5, 3)
    lat = np.linspace(0.0, 1e5, 3)
    dep = np.linspace(0.0, 3000.0, nz)
    data = np.zeros((1, 3, nz, 3, 3))
    data[0, 2] = w
    return lon, lat, dep, data


def test_age_counts_steps_and_deletes_at_max_age():
    lon, lat, dep, data = _still_3d()
    T = np.stack([np.full((31, 3, 3), 7.0)])
    f = O.Field(lon, lat, dep, np.zeros(1), data, tracers=(T,))
    for dt in (3600.0, -3600.0):
        st = _state(3, [5e4] * 3, [5e4] * 3, [100.0] * 3)
        age = np.array([0.0, 0.0, 5 * 3600.0])
        k = O.Kernel(O.RK4, O.AGE, max_age=10.5 * 3600.0)
        done = _run(f, k, st, dt, np.sign(dt) * 20 * 3600.0, age=age)
        # ages 0, 0 and 5 h: deleted after 11, 11 and 6 steps, each keeping its step
        np.testing.assert_array_equal(st["step"], [11, 11, 6])
        np.testing.assert_array_equal(age, [11 * 3600.0, 11 * 3600.0, 11 * 3600.0])
        np.testing.assert_array_equal(st["status"], [O.DELETED] * 3)
        np.testing.assert_array_equal(st["time"], np.sign(dt) * np.array([11, 11, 6]) * 3600.0)
        assert done == 28
    # a shortened last step adds its own length
    st = _state(1, [5e4], [5e4], [100.0])
    age = np.zeros(1)
    _run(f, O.Kernel(O.EULER, O.AGE, max_age=DAY), st, 3600.0, 2.5 * 3600.0, age=age)
    assert age[0] == 2.5 * 3600.0 and st["status"][0] == 0


def test_settle_and_age_two_phase_backward_closed_form():
    """The backward foraminifera run of Sect. 3 in a still ocean: from the
    floor at 2440 m the particle rises (backward in time) at the sinking speed
    of 200 m/day until it reaches its dwelling depth of 50 m, then holds that
    depth (even against a vertical velocity) while its age counts, and is
    deleted when the age reaches the 30-day lifespan."""
    w_sink = 200.0 / DAY
    for W in (0.0, 1e-4):
        lon, lat, dep, data = _still_3d(w=W)
        f = O.Field(lon, lat, dep, np.zeros(1), data)
        k = O.Kernel(O.EULER, O.SETTLE | O.AGE, w_sink=w_sink, dwell_depth=50.0,
                     max_age=30 * DAY)
        st = _state(1, [5e4], [5e4], [2440.0])
        age = np.zeros(1)
        dt = -3600.0
        # phase 1 by closed form: depth after m steps = 2440 - m * 200/24 (+ W), until 50 m
        rate = w_sink * 3600.0 + W * 3600.0
        m_reach = int(np.ceil((2440.0 - 50.0) / rate))
        _run(f, k, st, dt, dt * (m_reach - 1), age=age)
        assert st["depth"][0] > 50.0 and age[0] == 0.0
        assert abs(st["depth"][0] - (2440.0 - (m_reach - 1) * rate)) < 1e-9
        _run(f, k, st, dt, dt * m_reach, age=age)
        assert st["depth"][0] == 50.0 and age[0] == 0.0
        # phase 2: 720 hourly steps at 50 m, then deleted with its age at 30 days
        _run(f, k, st, dt, -100 * DAY, age=age)
        assert st["status"][0] == O.DELETED
        assert st["depth"][0] == 50.0
        assert age[0] == 30 * DAY
        assert st["step"][0] == m_reach + 720
        assert st["time"][0] == dt * (m_reach + 720)


def test_sample_behaviour_records_the_field_at_the_new_state():
    """SAMPLE stores the scalar field at the step's new position and time:
    in a uniform flow with a field linear in space and time, the variable
    equals the closed form at the particle's final position and time; a NaN
    region gives NaN without deleting the particle."""
    lon = np.linspace(0.0, 2e5, 21)
    lat = np.linspace(0.0, 2e5, 21)
    times = np.array([0.0, DAY, 2 * DAY])
    data = np.zeros((3, 2, 1, 21, 21))
    data[:, 0] = 0.5
    data[:, 1] = -0.2
    L, A = np.meshgrid(lon, lat, indexing="xy")
    T = np.stack([(4.0 + 1e-5 * L + 2e-5 * A + 1e-5 * t)[None] for t in times])
    T[:, :, 13:, 15:] = np.nan
    f = O.Field(lon, lat, np.zeros(1), times, data, tracers=(T,))
    st = _state(3, [1e4, 5e4, 1.3e5], [1.5e5, 1e5, 1.49e5], [0.0] * 3)
    var = np.full((1, 3), -1.0)
    _run(f, O.Kernel(O.RK4, O.SAMPLE), st, 1800.0, 0.75 * DAY, var=var)
    want = 4.0 + 1e-5 * st["lon"] + 2e-5 * st["lat"] + 1e-5 * st["time"]
    np.testing.assert_allclose(var[0, :2], want[:2], rtol=1e-13)
    assert st["status"][2] == 0 and np.isnan(var[0, 2])
    with pytest.raises(ValueError):
        _run(f, O.Kernel(O.RK4, O.SAMPLE), _state(1, [1e4], [1e4], [0.0]), 1800.0, DAY)
