"""Parity of the CUDA library with the FP64 oracle on the same seeded inputs.

FP64 path: within 1e-9 relative (relative to max(|x|, axis span)), deleted
sets equal; in practice the flat-mesh cases are bit-identical because both
sides carry out the same operations in the same order.  FP32 / FP16 / BF16
paths: within a stated number of grid cells.
"""
import numpy as np
import pytest

import oracle as O
import synth
from tests.helpers import (DAY, assert_close_positions, cell_error, gpu_run, oracle_field,
                           oracle_run)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1707_05163_gb300 as pg
    pg.load()
    return pg


def _outputs_match(g, o, tol, what):
    gk = sorted(k for k in g if not isinstance(k, str))
    ok = sorted(k for k in o if not isinstance(k, str))
    assert len(gk) == len(ok), (gk, ok)
    for a, b in zip(gk, ok):
        assert abs(a - b) <= 1e-6 * max(1.0, abs(b))
        assert_close_positions(g[a], o[b], tol, f"{what} t={b}")
    assert_close_positions(g["final"], o["final"], tol, f"{what} final")
    np.testing.assert_array_equal(g["final"]["step"], o["final"]["step"])
    np.testing.assert_array_equal(g["final"]["time"], o["final"]["time"])


def _tol64(spec):
    span = lambda a: max(abs(a[0]), abs(a[-1]), a[-1] - a[0]) if len(a) > 1 else 1.0
    return dict(lon=1e-9 * span(spec.lon), lat=1e-9 * span(spec.lat), depth=1e-9 * span(spec.depth))


# ---------------------------------------------------------------- FP64 path

def test_stommel_gyre_fp64_full_size(pg):
    """Steady 2-D gyre, 201x201 FP64, 1e4 particles, dt 1 h, 30 days, daily output."""
    spec = synth.stommel_gyre()
    L = 1e6
    rng = np.random.default_rng(1)
    lon = rng.uniform(0.05 * L, 0.95 * L, 10000)
    lat = rng.uniform(0.05 * L, 0.95 * L, 10000)
    o = oracle_run(oracle_field(spec), lon, lat, None, 0.0, 3600.0, 30 * DAY, DAY)
    fs = pg.FieldSet.from_spec(spec, storage="f64")
    ps = pg.ParticleSet(fs, lon, lat, pos="f64")
    g = gpu_run(ps, pg.Kernel("rk4"), 30 * DAY, 3600.0, DAY)
    assert g["steps"] == o["steps"] == 10000 * 720
    _outputs_match(g, o, _tol64(spec), "gyre")
    # flat mesh, same operation order: bit-identical
    np.testing.assert_array_equal(g["final"]["lon"], o["final"]["lon"])
    np.testing.assert_array_equal(g["final"]["lat"], o["final"]["lat"])


@pytest.mark.parametrize("case", ["rotation", "oscillating", "eddy", "peninsula", "zonal_sphere"])
def test_idealised_flows_fp64(pg, case):
    if case == "rotation":
        spec = synth.solid_body_rotation()
        lon, lat = np.zeros(4), np.array([1e3, 2e3, 3e3, 4e3])
        dt, T, out = 300.0, DAY, 3600.0
    elif case == "oscillating":
        spec = synth.oscillating_flow()
        lon, lat = np.linspace(-5e3, 5e3, 20), np.zeros(20)
        dt, T, out = 300.0, 4 * DAY, 3 * 3600.0
    elif case == "eddy":
        spec = synth.decaying_eddy()
        lon, lat = np.array([1e3, -3e3, 5e3]), np.array([2e3, 4e3, -1e3])
        dt, T, out = 300.0, 4 * DAY, 3600.0
    elif case == "peninsula":
        spec = synth.peninsula()
        lon, lat = np.full(20, 1000.0), np.linspace(26e3, 52e3, 20)
        dt, T, out = 300.0, DAY, 3600.0
    else:
        spec = synth.zonal_flow_sphere()
        lon, lat = np.zeros(31), np.arange(-45.0, 45.1, 3.0)
        dt, T, out = 300.0, 57 * DAY, DAY
    o = oracle_run(oracle_field(spec), lon, lat, None, 0.0, dt, T, out)
    fs = pg.FieldSet.from_spec(spec, storage="f64")
    ps = pg.ParticleSet(fs, lon, lat, pos="f64")
    g = gpu_run(ps, pg.Kernel("rk4"), T, dt, out)
    _outputs_match(g, o, _tol64(spec), case)


def test_brownian_fp64_bit_exact_random_stream(pg):
    """Brownian motion (Sect. 4.2.7): the Philox stream is the same on both
    sides, so positions agree to the rounding of log/cos/sin."""
    spec = synth.zero_field()
    n = 20000
    lon, lat = np.zeros(n), np.zeros(n)
    ids = np.arange(n, dtype=np.uint64) * 7919 + 3
    o = oracle_run(oracle_field(spec), lon, lat, None, 0.0, 300.0, DAY, 0.0,
                   behaviours=("brownian",), kh=100.0, seed=42, ids=ids)
    fs = pg.FieldSet.from_spec(spec, storage="f64")
    ps = pg.ParticleSet(fs, lon, lat, ids=ids, pos="f64", seed=42)
    g = gpu_run(ps, pg.Kernel("rk4", ("brownian",), kh=100.0), DAY, 300.0)
    np.testing.assert_array_equal(g["final"]["id"], np.sort(ids))
    order = np.argsort(ids)
    for ax in ("lon", "lat"):
        np.testing.assert_allclose(g["final"][ax], o["final"][ax][order], rtol=0, atol=1e-9 * 3e4)
    var = np.var(g["final"]["lon"])
    assert abs(var / (2 * 100.0 * DAY) - 1) < 4 * np.sqrt(2.0 / n)


def test_sinking_and_depth_deletion_3d_fp64(pg):
    rng = np.random.default_rng(9)
    spec, _ = synth.linear_field(rng, nx=9, ny=8, nz=7, nt=4, nfields=3)
    spec.data *= 1e-3
    n = 500
    lon = rng.uniform(spec.lon[1], spec.lon[-2], n)
    lat = rng.uniform(spec.lat[1], spec.lat[-2], n)
    dep = rng.uniform(spec.depth[0], spec.depth[-1], n)
    T = spec.times[-1] - 1.0
    o = oracle_run(oracle_field(spec), lon, lat, dep, 0.0, 600.0, T, 6 * 3600.0,
                   behaviours=("sink",), w_sink=2e-3)
    fs = pg.FieldSet.from_spec(spec, storage="f64")
    ps = pg.ParticleSet(fs, lon, lat, dep, pos="f64")
    g = gpu_run(ps, pg.Kernel("rk4", ("sink",), w_sink=2e-3), T, 600.0, 6 * 3600.0)
    _outputs_match(g, o, _tol64(spec), "sinking")
    assert (o["final"]["status"] != 0).sum() > 10      # some left the domain


def test_backward_in_time_fp64(pg):
    spec = synth.decaying_eddy()
    lon, lat = np.array([1e3, -3e3, 5e3, 0.0]), np.array([2e3, 4e3, -1e3, 500.0])
    T0 = 3 * DAY
    o = oracle_run(oracle_field(spec), lon, lat, None, T0, -300.0, 2 * DAY, 6 * 3600.0)
    fs = pg.FieldSet.from_spec(spec, storage="f64")
    ps = pg.ParticleSet(fs, lon, lat, t0=T0, pos="f64")
    g = gpu_run(ps, pg.Kernel("rk4"), 2 * DAY, -300.0, 6 * 3600.0)
    _outputs_match(g, o, _tol64(spec), "backward")


def test_euler_and_ragged_sizes_fp64(pg):
    spec = synth.stommel_gyre(n=51)
    rng = np.random.default_rng(2)
    for n in (1, 31, 257, 1000):
        lon = rng.uniform(5e4, 9.5e5, n)
        lat = rng.uniform(5e4, 9.5e5, n)
        o = oracle_run(oracle_field(spec), lon, lat, None, 0.0, 1800.0, 2 * DAY + 900.0,
                       scheme="euler")
        fs = pg.FieldSet.from_spec(spec, storage="f64")
        ps = pg.ParticleSet(fs, lon, lat, pos="f64")
        g = gpu_run(ps, pg.Kernel("euler"), 2 * DAY + 900.0, 1800.0)
        assert_close_positions(g["final"], o["final"], _tol64(spec), f"euler n={n}")
        assert (g["final"]["time"] == 2 * DAY + 900.0).all()


@pytest.mark.parametrize("nt", [1, 3])
def test_nan_islands_delete_with_nan_status(pg, nt):
    """NaN nodes (land) make every cell that touches them return NaN; a stage
    sampling there deletes the particle with PG_NAN and keeps its last valid
    state.  FP64 matches the oracle bit for bit (flat mesh); the FP32 forms
    report the same statuses (steady and time-dependent fields)."""
    import dataclasses
    base = synth.stommel_gyre(n=61)
    amp = [1.0, 1.3, 0.7][:nt]
    data = np.concatenate([base.data * a for a in amp], axis=0).copy()
    rng = np.random.default_rng(5)
    for _ in range(25):
        i, j = rng.integers(3, 58, 2)
        data[:, :, 0, j:j + 2, i:i + 3] = np.nan
    times = np.arange(nt) * 5 * DAY if nt > 1 else np.zeros(1)
    spec = dataclasses.replace(base, data=data, times=times)
    n = 4000
    lon = rng.uniform(2e4, 9.8e5, n)
    lat = rng.uniform(2e4, 9.8e5, n)
    dt, T = 3600.0, 8 * DAY
    o = oracle_run(oracle_field(spec), lon, lat, None, 0.0, dt, T)
    st = o["final"]["status"]
    assert (st == 3).sum() > 200 and (st == 0).sum() > 1000
    fs64 = pg.FieldSet.from_spec(spec, storage="f64")
    g = gpu_run(pg.ParticleSet(fs64, lon, lat, pos="f64"), pg.Kernel("rk4"), T, dt)
    for k in ("lon", "lat", "status", "step", "time"):
        np.testing.assert_array_equal(g["final"][k], o["final"][k], err_msg=k)
    fs32 = pg.FieldSet.from_spec(spec, storage="f32")
    for pos in ("f32", "cell"):
        g = gpu_run(pg.ParticleSet(fs32, lon.astype(np.float32), lat.astype(np.float32), pos=pos),
                    pg.Kernel("rk4"), T, dt)
        gs = g["final"]["status"]
        assert set(np.unique(gs)) <= {0, 1, 3}
        assert np.mean(gs == st) > 0.99, (pos, np.mean(gs == st))
        alive = (gs == 0) & (st == 0)
        e = cell_error(g["final"], o["final"], spec, periodic=False)[alive]
        assert np.mean(e) < 1e-3, (pos, np.mean(e))


def test_empty_particle_set(pg):
    fs = pg.FieldSet.from_spec(synth.stommel_gyre(n=11), storage="f64")
    ps = pg.ParticleSet(fs, np.zeros(0), np.zeros(0), pos="f64")
    assert ps.execute(pg.Kernel("rk4"), DAY, 3600.0) == 0
    assert len(ps) == 0


# --------------------------------------------------------- reduced paths

def _small_global(nt=4, nz=8, res=2.0, seed=12):
    gf = synth.GlobalField(res_deg=res, nz=nz, nt=nt, seed=seed, kmax=20, period=nt * DAY)
    return gf, gf.spec(materialise=True)


def test_fp32_global_3d_within_cells(pg):
    gf, spec = _small_global()
    lon, lat, dep = synth.uniform_particles(4000, 5, (0, 360), (-70, 70), (6.0, 1000.0),
                                            dtype=np.float32)
    T = 3 * DAY
    o = oracle_run(oracle_field(spec), lon, lat, dep, 0.0, 1800.0, T)
    fs = pg.FieldSet.from_spec(spec, storage="f32")
    ps = pg.ParticleSet(fs, lon, lat, dep, pos="f32")
    g = gpu_run(ps, pg.Kernel("rk4"), T, 1800.0)
    np.testing.assert_array_equal(g["final"]["status"], o["final"]["status"])
    alive = o["final"]["status"] == 0
    e = cell_error(g["final"], o["final"], spec)[alive]
    assert np.mean(e) < 1e-3 and np.max(e) < 2e-2, (np.mean(e), np.max(e))
    assert g["steps"] == o["steps"]


@pytest.mark.parametrize("geo", ["flat", "sphere_regional", "sphere_coarse_lat"])
def test_fp32_each_mesh_geometry(pg, geo):
    """The FP32 kernels are compiled once per geometry (flat; spherical;
    spherical with a periodic zonal boundary).  Each kind against the oracle,
    the spherical ones on a 1-degree regional grid and on a coarse global grid
    with 12-degree cells."""
    import dataclasses
    if geo == "flat":
        spec = synth.stommel_gyre(n=101)
        rng = np.random.default_rng(31)
        lon = rng.uniform(1e5, 9e5, 3000).astype(np.float32)
        lat = rng.uniform(1e5, 9e5, 3000).astype(np.float32)
        dt, T = 3600.0, 20 * DAY
    else:
        gf, spec = _small_global(nz=1, res=12.0 if geo == "sphere_coarse_lat" else 1.0)
        if geo == "sphere_regional":
            keep = spec.lon <= 120.0
            spec = dataclasses.replace(spec, lon=spec.lon[keep], data=spec.data[..., keep],
                                       periodic_lon=False)
        lon, lat, _ = synth.uniform_particles(3000, 11, (spec.lon[0], spec.lon[-1]),
                                              (spec.lat[0], spec.lat[-1]), dtype=np.float32)
        dt, T = 1800.0, 3 * DAY
    o = oracle_run(oracle_field(spec), lon, lat, None, 0.0, dt, T)
    fs = pg.FieldSet.from_spec(spec, storage="f32")
    ps = pg.ParticleSet(fs, lon, lat, pos="f32")
    g = gpu_run(ps, pg.Kernel("rk4"), T, dt)
    np.testing.assert_array_equal(g["final"]["status"], o["final"]["status"])
    alive = o["final"]["status"] == 0
    assert alive.sum() > 1000
    e = cell_error(g["final"], o["final"], spec, periodic=spec.periodic_lon)[alive]
    assert np.mean(e) < 1e-3 and np.max(e) < 2e-2, (np.mean(e), np.max(e))
    assert g["steps"] == o["steps"]


@pytest.mark.parametrize("pos", ["f32", "cell"])
def test_fp32_metres_to_degrees_on_the_sphere(pg, pos):
    """Uniform 1 m/s eastward flow on the sphere (Sect. 4.2.2): one RK4 step of
    one day moves a particle by u dt / (1852 * 60 * cos(lat)) degrees of
    longitude exactly (every stage sees the same velocity), so the FP32 step
    pins the FP32 cos(lat) and the metres-to-degrees conversion to a few ulps
    from the equator to 80 degrees."""
    spec = synth.zonal_flow_sphere()
    lat = np.linspace(-79.75, 79.75, 320)
    lon = np.full(lat.shape, 0.5)
    fs = pg.FieldSet.from_spec(spec, storage="f32")
    ps = pg.ParticleSet(fs, lon.astype(np.float32), lat.astype(np.float32), pos=pos)
    ps.execute(pg.Kernel("rk4"), DAY, DAY)
    g = ps.get()
    lat32 = lat.astype(np.float32).astype(np.float64)
    want = 0.5 + DAY / (1852.0 * 60.0 * np.cos(np.deg2rad(lat32)))
    rel = np.abs(g["lon"] - want) / (want - 0.5)
    assert (g["status"] == 0).all()
    np.testing.assert_array_equal(g["lat"], lat32)
    assert rel.max() < 3e-6, rel.max()


@pytest.mark.parametrize("storage,kind", [("f16", 0), ("bf16", 1)])
def test_quantised_storage_scales_and_trajectories(pg, storage, kind):
    gf, spec = _small_global(nz=1, res=1.0)
    fs = pg.FieldSet.from_spec(spec, storage=storage)
    data_q = np.empty(spec.data.shape, dtype=np.float64)
    for s in range(spec.nt):
        for f in range(spec.data.shape[1]):
            q, sc = O.quantise(spec.data[s, f], kind)
            assert fs.scale(s, f) == sc
            data_q[s, f] = O.dequantise(q, kind, sc)
    lon, lat, dep = synth.uniform_particles(3000, 6, (0, 360), (-70, 70), dtype=np.float32)
    T = 2 * DAY
    o = oracle_run(oracle_field(spec, data_q), lon, lat, None, 0.0, 3600.0, T)
    ps = pg.ParticleSet(fs, lon, lat, pos="f32")
    g = gpu_run(ps, pg.Kernel("rk4"), T, 3600.0)
    alive = o["final"]["status"] == 0
    e = cell_error(g["final"], o["final"], spec)[alive]
    assert np.mean(e) < 1e-3, np.mean(e)


def test_streamed_equals_resident(pg):
    gf, spec = _small_global(nt=5)
    lon, lat, dep = synth.uniform_particles(2000, 7, (0, 360), (-70, 70), (6.0, 900.0),
                                            dtype=np.float32)
    T = 4.5 * DAY
    res = []
    for mode in ("resident", "ptrs", "callback", "ring6"):
        if mode == "resident":
            fs = pg.FieldSet.from_spec(spec, storage="f32")
        else:
            fs = pg.FieldSet(spec.lon, spec.lat, spec.depth, mesh="spherical", periodic_lon=True,
                             nfields=spec.data.shape[1], storage="f32")
            fs.set_times(spec.times, spec.period)
            if mode == "ring6":
                fs.set_ring(6)
                fs.stream([spec.data[s] for s in range(spec.nt)])
            elif mode == "ptrs":
                fs.stream([spec.data[s] for s in range(spec.nt)])
            else:
                fs.stream(callback=lambda s, out: out.__setitem__(Ellipsis, spec.data[s]))
        ps = pg.ParticleSet(fs, lon, lat, dep, pos="f32")
        if mode == "ring6":       # launches of up to two days across snapshot times, two
                                  # snapshots prefetched
            ps.set_tune(block=128, resort_steps=0, chunk_steps=200)
        res.append(gpu_run(ps, pg.Kernel("rk4"), T, 1800.0, 2.25 * DAY if mode == "ring6" else DAY))
    for r in res[1:]:
        for k in ("lon", "lat", "depth", "status", "time"):
            np.testing.assert_array_equal(r["final"][k], res[0]["final"][k])


def test_resort_and_checkpoint_are_invisible(pg, tmp_path):
    gf, spec = _small_global()
    lon, lat, dep = synth.uniform_particles(5000, 8, (0, 360), (-75, 75), (6.0, 900.0),
                                            dtype=np.float32)
    fs = pg.FieldSet.from_spec(spec, storage="f32")
    K = pg.Kernel("rk4", ("brownian",), kh=10.0)
    a = pg.ParticleSet(fs, lon, lat, dep, pos="f32", seed=3)
    a.execute(K, 2 * DAY, 1800.0)
    ref = a.get()
    b = pg.ParticleSet(fs, lon, lat, dep, pos="f32", seed=3)
    b.set_tune(block=128, resort_steps=7, chunk_steps=5)
    b.execute(K, DAY, 1800.0)
    path = tmp_path / "ck.bin"
    b.save(path)
    c = pg.ParticleSet.restore(fs, path)
    c.set_tune(resort_steps=11)
    c.execute(K, DAY, 1800.0)
    got = c.get()
    for k in ("lon", "lat", "depth", "time", "step", "status", "id"):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    m = c.moments()
    alive = got["status"] == 0
    assert m[0] == alive.sum()
    np.testing.assert_allclose(m[1:4], [got[k][alive].sum() for k in ("lon", "lat", "depth")],
                               rtol=1e-12)
    np.testing.assert_allclose(m[4:7], [(got[k][alive] ** 2).sum() for k in ("lon", "lat", "depth")],
                               rtol=1e-12)


def test_error_conventions(pg):
    spec = synth.decaying_eddy(days=1.0)
    fs = pg.FieldSet.from_spec(spec, storage="f64")
    ps = pg.ParticleSet(fs, np.array([0.0]), np.array([0.0]), pos="f64")
    before = ps.get()
    with pytest.raises(pg.PGError) as e:
        ps.execute(pg.Kernel("rk4"), 2 * DAY, 300.0)
    assert e.value.code == -4          # outside the field's time range
    after = ps.get()
    for k in before:
        np.testing.assert_array_equal(before[k], after[k])
    with pytest.raises(pg.PGError) as e:
        fs.load_snapshot(10 ** 6, spec.data[0])
    assert e.value.code == -1
    gf, gspec = _small_global(nt=3)
    fs2 = pg.FieldSet(gspec.lon, gspec.lat, gspec.depth, mesh="spherical", periodic_lon=True,
                      nfields=3, storage="f32")
    fs2.set_times(gspec.times, gspec.period)

    def bad(s, out):
        if s == 2:
            raise IOError("snapshot unreadable")
        out[...] = gspec.data[s]
    fs2.stream(callback=bad)
    ps2 = pg.ParticleSet(fs2, np.array([10.0]), np.array([5.0]), np.array([50.0]))
    with pytest.raises(pg.PGError) as e:
        ps2.execute(pg.Kernel("rk4"), 2.5 * DAY, 1800.0)
    assert e.value.code == -5
