"""Parity of the precision form (cell index + FP32 offset positions; FP32,
FP16 or BF16 field storage) with the FP64 oracle.

The oracle runs in physical FP64 coordinates on the same stored field values
(dequantised, for FP16/BF16), so the comparison isolates the error of the
reduced position arithmetic.  Tolerance: mean position error below 1e-3 cell
and maximum below 1e-2 cell; deleted sets equal.
"""
import numpy as np
import pytest

import oracle as O
import synth
from tests.helpers import DAY, cell_error, gpu_run, oracle_field, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1707_05163_gb300 as pg
    pg.load()
    return pg


def _surface(res=1.0, nt=4, seed=21):
    gf = synth.GlobalField(res_deg=res, nz=1, nt=nt, seed=seed, kmax=30, period=nt * DAY)
    return gf.spec(materialise=True)


def _dequantised(spec, kind):
    out = np.empty(spec.data.shape, dtype=np.float64)
    for s in range(spec.nt):
        for f in range(spec.data.shape[1]):
            q, sc = O.quantise(spec.data[s, f], kind)
            out[s, f] = O.dequantise(q, kind, sc)
    return out


def test_cell_roundtrip_of_positions(pg):
    spec = _surface()
    lon, lat, _ = synth.uniform_particles(5000, 3, (-20, 400), (-85, 85))
    lon = np.concatenate([lon, spec.lon[[0, 5, -1]], [359.5]])
    lat = np.concatenate([lat, spec.lat[[0, 7, -1]], [spec.lat[-1]]])
    fs = pg.FieldSet.from_spec(spec, storage="f32")
    ps = pg.ParticleSet(fs, lon, lat, pos="cell")
    got = ps.get()
    dx = spec.lon[1] - spec.lon[0]
    dlon = (got["lon"] - lon + 180.0) % 360.0 - 180.0
    assert np.max(np.abs(dlon)) / dx < 1e-6
    assert np.max(np.abs(got["lat"] - lat)) / dx < 1e-6
    assert (got["lon"] >= 0.0).all() and (got["lon"] < 360.0).all()


@pytest.mark.parametrize("storage,kind", [("f32", None), ("f16", 0), ("bf16", 1)])
def test_cell_form_against_oracle(pg, storage, kind):
    spec = _surface()
    data = spec.data if kind is None else _dequantised(spec, kind)
    lon, lat, _ = synth.uniform_particles(4000, 4, (0, 360), (-75, 75))
    T = 3 * DAY
    o = oracle_run(oracle_field(spec, data), lon, lat, None, 0.0, 3600.0, T)
    fs = pg.FieldSet.from_spec(spec, storage=storage)
    ps = pg.ParticleSet(fs, lon, lat, pos="cell")
    g = gpu_run(ps, pg.Kernel("rk4"), T, 3600.0)
    np.testing.assert_array_equal(g["final"]["status"], o["final"]["status"])
    alive = o["final"]["status"] == 0
    e = cell_error(g["final"], o["final"], spec)[alive]
    assert np.mean(e) < 1e-3 and np.max(e) < 1e-2, (np.mean(e), np.max(e))
    assert g["steps"] == o["steps"]


def test_cell_form_brownian_same_random_stream(pg):
    spec = _surface(nt=3)
    data = _dequantised(spec, 0)
    lon, lat, _ = synth.uniform_particles(3000, 5, (0, 360), (-60, 60))
    T = 2 * DAY
    o = oracle_run(oracle_field(spec, data), lon, lat, None, 0.0, 3600.0, T,
                   behaviours=("brownian",), kh=10.0, seed=77)
    fs = pg.FieldSet.from_spec(spec, storage="f16")
    ps = pg.ParticleSet(fs, lon, lat, pos="cell", seed=77)
    g = gpu_run(ps, pg.Kernel("rk4", ("brownian",), kh=10.0), T, 3600.0)
    alive = o["final"]["status"] == 0
    e = cell_error(g["final"], o["final"], spec)[alive]
    assert np.mean(e) < 1e-3 and np.max(e) < 1e-2, (np.mean(e), np.max(e))


def test_cell_form_flat_gyre_and_sinking_3d(pg):
    spec = synth.stommel_gyre(n=101)
    spec.data = spec.data.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(6)
    lon = rng.uniform(5e4, 9.5e5, 2000)
    lat = rng.uniform(5e4, 9.5e5, 2000)
    o = oracle_run(oracle_field(spec), lon, lat, None, 0.0, 3600.0, 10 * DAY)
    fs = pg.FieldSet.from_spec(spec, storage="f32")
    ps = pg.ParticleSet(fs, lon, lat, pos="cell")
    g = gpu_run(ps, pg.Kernel("rk4"), 10 * DAY, 3600.0)
    e = cell_error(g["final"], o["final"], spec, periodic=False)
    assert np.mean(e) < 1e-3 and np.max(e) < 1e-2, (np.mean(e), np.max(e))
    # 3-D uniform depth axis, sinking through the bottom
    gf = synth.GlobalField(res_deg=4.0, nz=6, nt=3, seed=2, kmax=8, period=3 * DAY)
    s3 = gf.spec(materialise=True)
    s3.depth = np.linspace(5.0, 505.0, 6)
    lo3, la3, de3 = synth.uniform_particles(2000, 8, (0, 360), (-60, 60), (10.0, 480.0))
    o3 = oracle_run(oracle_field(s3), lo3, la3, de3, 0.0, 1800.0, DAY, behaviours=("sink",),
                    w_sink=2e-3)
    fs3 = pg.FieldSet.from_spec(s3, storage="f32")
    ps3 = pg.ParticleSet(fs3, lo3, la3, de3, pos="cell")
    g3 = gpu_run(ps3, pg.Kernel("rk4", ("sink",), w_sink=2e-3), DAY, 1800.0)
    np.testing.assert_array_equal(g3["final"]["status"], o3["final"]["status"])
    alive = o3["final"]["status"] == 0
    e3 = cell_error(g3["final"], o3["final"], s3)[alive]
    assert np.mean(e3) < 1e-3 and np.max(e3) < 1e-2, (np.mean(e3), np.max(e3))
    assert (~alive).sum() > 0


def test_cell_form_resort_and_checkpoint(pg, tmp_path):
    spec = _surface(nt=3)
    lon, lat, _ = synth.uniform_particles(6000, 9, (0, 360), (-70, 70))
    fs = pg.FieldSet.from_spec(spec, storage="bf16")
    K = pg.Kernel("rk4", ("brownian",), kh=5.0)
    a = pg.ParticleSet(fs, lon, lat, pos="cell", seed=11)
    a.execute(K, 2 * DAY, 3600.0)
    ref = a.get()
    b = pg.ParticleSet(fs, lon, lat, pos="cell", seed=11)
    b.set_tune(block=64, resort_steps=5, chunk_steps=7)
    b.execute(K, DAY, 3600.0)
    b.save(tmp_path / "c.bin")
    c = pg.ParticleSet.restore(fs, tmp_path / "c.bin")
    c.execute(K, DAY, 3600.0)
    got = c.get()
    for k in ("lon", "lat", "time", "step", "status", "id"):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    m = c.moments()
    alive = got["status"] == 0
    np.testing.assert_allclose(m[1:3], [got["lon"][alive].sum(), got["lat"][alive].sum()],
                               rtol=1e-12)


def test_cell_form_needs_uniform_axes(pg):
    rng = np.random.default_rng(1)
    spec, _ = synth.linear_field(rng, nz=4, nt=1, nfields=3)
    fs = pg.FieldSet.from_spec(spec, storage="f32")
    with pytest.raises(pg.PGError) as e:
        pg.ParticleSet(fs, spec.lon[[1]], spec.lat[[1]], spec.depth[[1]], pos="cell")
    assert e.value.code == -8
