"""Trajectory output through the pinned ring (the ParticleFile of Sect. 3):
complete records and the indexed form against the oracle at every output
time, the particle variables carried along, and the error convention of a
failing hook."""
import numpy as np
import pytest

import oracle as O
import synth
from tests.helpers import DAY, oracle_field, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1707_05163_gb300 as pg
    pg.load()
    return pg


def _gyre_case(n, seed):
    """The Stommel gyre with an eastward drift of 0.3 m/s added, so that
    particles leave through the eastern boundary during the run."""
    spec = synth.stommel_gyre(n=101)
    spec.data = spec.data.copy()
    spec.data[:, 0] += 0.3
    rng = np.random.default_rng(seed)
    L = 1e6
    lon = rng.uniform(0.0, L, n)
    lat = rng.uniform(0.0, L, n)
    return spec, lon, lat


@pytest.mark.parametrize("indexed", [False, True])
def test_records_against_oracle_fp64(pg, indexed):
    """200,003 particles (13 compaction tiles and a ragged one), output every
    12 h for 5 days with 1 h steps and launches of 7 steps: every record equals
    the oracle's state at that time (FP64, flat mesh: bit for bit); the
    indexed form holds exactly the particles alive at that time and those
    deleted since the previous output."""
    n = 200_003
    spec, lon, lat = _gyre_case(n, 3)
    out_dt, T = 0.5 * DAY, 5 * DAY
    o = oracle_run(oracle_field(spec), lon, lat, None, 0.0, 3600.0, T, out_dt)
    fs = pg.FieldSet.from_spec(spec, storage="f64")
    ps = pg.ParticleSet(fs, lon, lat, pos="f64")
    ps.set_tune(block=128, resort_steps=9, chunk_steps=7)
    got = {}
    steps = ps.execute_records(pg.Kernel("rk4"), T, 3600.0, out_dt,
                               lambda t, r: got.__setitem__(t, r), indexed=indexed)
    assert steps == o["steps"]
    times = sorted(k for k in o if not isinstance(k, str))
    assert sorted(got) == times
    prev = np.zeros(n, np.uint8)
    for t in times:
        r, ref = got[t], o[t]
        order = np.argsort(r["id"])
        ids = r["id"][order].astype(np.int64)
        if indexed:
            want = np.nonzero((ref["status"] == 0) | (prev == 0))[0]
        else:
            want = np.arange(n)
        np.testing.assert_array_equal(ids, want, err_msg=f"rows at t={t}")
        for k in ("lon", "lat", "status"):
            np.testing.assert_array_equal(r[k][order], ref[k][want], err_msg=f"{k} t={t}")
        prev = ref["status"]
    final = o["final"]["status"]
    assert (final != 0).sum() > 10_000 and (final == 0).sum() > 100_000


def test_records_carry_variables_and_cell_positions(pg):
    """Records of the cell form (positions turned back into lon/lat) and of
    the worked example's variables: the last record equals the particle set's
    final state and variables."""
    gf = synth.GlobalField(res_deg=2.0, nz=1, nt=3, seed=17, kmax=20, period=3 * DAY)
    spec = gf.spec(materialise=True)
    lon, lat, _ = synth.uniform_particles(50_000, 3, (0, 360), (-80, 80), dtype=np.float32)
    fs = pg.FieldSet.from_spec(spec, storage="f32")
    ps = pg.ParticleSet(fs, lon, lat, pos="cell")
    got = {}
    ps.execute_records(pg.Kernel("rk4"), 2 * DAY, 1800.0, DAY,
                       lambda t, r: got.__setitem__(t, r), indexed=False)
    assert sorted(got) == [DAY, 2 * DAY]
    g = ps.get()
    r = got[2 * DAY]
    o = np.argsort(r["id"])
    for k in ("lon", "lat", "status"):
        np.testing.assert_array_equal(r[k][o], g[k], err_msg=k)
    # variables: age and a sampled temperature on FP32 positions
    rng = np.random.default_rng(5)
    s3, _ = synth.linear_field(rng, nx=12, ny=10, nz=6, nt=3, nfields=3)
    s3.data *= 1e-3
    temp = synth.temperature(s3.lon, s3.lat, s3.depth, s3.times, seed=2)
    f3 = pg.FieldSet.from_spec(s3, storage="f32")
    f3.add_scalar("T")
    for s in range(s3.nt):
        f3.load_scalar(0, s, temp[s])
    f3.add_constant("max_age", 1.5 * DAY)
    m = 5000
    p3 = pg.ParticleSet(f3, rng.uniform(s3.lon[1], s3.lon[-2], m),
                        rng.uniform(s3.lat[1], s3.lat[-2], m),
                        rng.uniform(s3.depth[1], s3.depth[-2], m), pos="f32")
    recs = {}
    p3.execute_records(pg.Kernel("rk4", ("age", "sample")), 2 * DAY, 900.0, 0.5 * DAY,
                       lambda t, r: recs.__setitem__(t, r), indexed=True)
    last = recs[2 * DAY]
    v = p3.get_variables()
    gs = p3.get()
    o = np.argsort(last["id"])
    ids = last["id"][o].astype(np.int64)
    # by the end every particle is deleted (age or domain): the last record
    # holds those deleted in its interval, with their final variables
    np.testing.assert_array_equal(last["age"][o], v["age"][ids])
    np.testing.assert_array_equal(last["vars"][0][o], v["vars"][0][ids])
    np.testing.assert_array_equal(last["status"][o], gs["status"][ids])
    seen = np.concatenate([recs[t]["id"] for t in sorted(recs)])
    assert len(np.unique(seen)) == m               # every particle appears
    assert (v["age"] <= 1.5 * DAY).all() and (gs["status"] == 4).sum() > 300


def test_failing_record_hook(pg):
    spec, lon, lat = _gyre_case(1000, 4)
    fs = pg.FieldSet.from_spec(spec, storage="f64")
    ps = pg.ParticleSet(fs, lon, lat, pos="f64")
    calls = []

    def hook(t, r):
        calls.append(t)
        return 1 if len(calls) == 2 else 0
    with pytest.raises(pg.PGError) as e:
        ps.execute_records(pg.Kernel("rk4"), 3 * DAY, 3600.0, 0.5 * DAY, hook)
    assert e.value.code == -5 and len(calls) == 2
    # the set can run on
    assert ps.execute(pg.Kernel("rk4"), DAY, 3600.0) > 0
