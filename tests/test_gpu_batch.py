"""Batched form: many releases of uneven size, dt, runtime and kernel in one
persistent launch per window, with and without a CUDA graph, autotuned or
fixed; checked against one execute per release and against the oracle."""
import numpy as np
import pytest

import synth
from tests.helpers import DAY, cell_error, oracle_field, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1707_05163_gb300 as pg
    pg.load()
    return pg


@pytest.fixture(scope="module")
def field():
    gf = synth.GlobalField(res_deg=2.0, nz=8, nt=5, seed=31, kmax=20, period=5 * DAY)
    return gf.spec(materialise=True)


def _releases(scale=1.0):
    # sizes straddle the re-sort threshold (65,536) and the tile size
    spec = [(70000, 600.0, 3.0, 0), (3000, 7200.0, 7.5, 1), (257, 1800.0, 2.0, 2),
            (90000, 3600.0, 5.0, 1), (1, 900.0, 1.0, 0), (12345, 2400.0, 6.0, 2)]
    out = []
    for r, (n, dt, days, kind) in enumerate(spec):
        out.append(synth.Release(max(1, int(n * scale)), dt, days * DAY, kind,
                                 kh=[0.0, 20.0, 0.0][kind], w_sink=[0.0, 0.0, 5e-4][kind],
                                 seed=100 + r))
    return out


def _kernel(pg, rel):
    if rel.kind == 0:
        return pg.Kernel("rk4")
    if rel.kind == 1:
        return pg.Kernel("rk4", ("brownian",), kh=rel.kh)
    return pg.Kernel("rk4", ("sink",), w_sink=rel.w_sink)


def _psets(pg, fs, rels):
    out = []
    for r, rel in enumerate(rels):
        lon, lat, dep = synth.uniform_particles(rel.n, rel.seed, (0, 360), (-70, 70), (6.0, 900.0),
                                                dtype=np.float32)
        out.append(pg.ParticleSet(fs, lon, lat, dep, pos="f32", seed=rel.seed,
                                  id_base=1_000_000 * r))
    return out


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_equals_one_execute_per_release(pg, field, use_graph):
    fs = pg.FieldSet.from_spec(field, storage="f32")
    rels = _releases()
    kernels = [_kernel(pg, r) for r in rels]
    batch = _psets(pg, fs, rels)
    steps, used = pg.execute_batch(batch, kernels, [r.runtime for r in rels],
                                   [r.dt for r in rels], tune=(128, 1), use_graph=use_graph)
    assert used == (128, 1)
    single = _psets(pg, fs, rels)
    total = 0
    for ps, k, r in zip(single, kernels, rels):
        total += ps.execute(k, r.runtime, r.dt)
    assert steps == total
    for a, b, r in zip(batch, single, rels):
        ga, gb = a.get(), b.get()
        np.testing.assert_array_equal(ga["id"], gb["id"])
        np.testing.assert_array_equal(ga["status"], gb["status"])
        np.testing.assert_array_equal(ga["step"], gb["step"])
        np.testing.assert_array_equal(ga["time"], gb["time"])
        # same FP32 operations in the same order: bit-identical positions
        for k in ("lon", "lat", "depth"):
            np.testing.assert_array_equal(ga[k], gb[k], err_msg=f"{k} {r}")
        ok = ga["status"] == 0
        assert (ga["time"][ok] == r.runtime).all()


def test_batch_autotuner_and_cache(pg, field, tmp_path):
    fs = pg.FieldSet.from_spec(field, storage="f32")
    rels = _releases(scale=0.5)
    kernels = [_kernel(pg, r) for r in rels]
    cache = tmp_path / "tune.txt"
    a = _psets(pg, fs, rels)
    s1, used1 = pg.execute_batch(a, kernels, [r.runtime for r in rels], [r.dt for r in rels],
                                 tune=None, tune_cache=cache)
    # candidates: never, every 1, 2 or 4 windows, or before the first window
    # only (an interval of at least five windows, the run's window count)
    assert used1[0] in (64, 128, 256) and (used1[1] in (0, 1, 2, 4) or used1[1] >= 5)
    assert cache.read_text().strip().endswith(f"{used1[0]} {used1[1]}")
    b = _psets(pg, fs, rels)
    s2, used2 = pg.execute_batch(b, kernels, [r.runtime for r in rels], [r.dt for r in rels],
                                 tune=None, tune_cache=cache)
    assert used2 == used1 and s2 == s1
    # the tuning trials ran on a saved copy: results equal a fixed-tune run
    c = _psets(pg, fs, rels)
    s3, _ = pg.execute_batch(c, kernels, [r.runtime for r in rels], [r.dt for r in rels],
                             tune=used1)
    assert s3 == s1
    for x, y in zip(a, c):
        gx, gy = x.get(), y.get()
        np.testing.assert_array_equal(gx["status"], gy["status"])
        ok = gx["status"] == 0
        assert np.max(cell_error(gx, gy, field)[ok], initial=0.0) < 1e-5


def test_batch_against_oracle(pg, field):
    fs = pg.FieldSet.from_spec(field, storage="f32")
    rels = _releases(scale=0.02)
    kernels = [_kernel(pg, r) for r in rels]
    batch = _psets(pg, fs, rels)
    starts = [p.get() for p in batch]
    pg.execute_batch(batch, kernels, [r.runtime for r in rels], [r.dt for r in rels],
                     tune=(64, 1))
    f = oracle_field(field)
    for ps, st0, r in zip(batch, starts, rels):
        beh = [(), ("brownian",), ("sink",)][r.kind]
        o = oracle_run(f, st0["lon"], st0["lat"], st0["depth"], 0.0, r.dt, r.runtime,
                       behaviours=beh, kh=r.kh, w_sink=r.w_sink, seed=r.seed, ids=st0["id"])
        g = ps.get()
        order = np.argsort(o["final"]["ids"])
        of = {k: v[order] for k, v in o["final"].items()}
        np.testing.assert_array_equal(g["status"], of["status"])
        ok = g["status"] == 0
        e = cell_error(g, of, field)[ok]
        assert e.size == 0 or (np.mean(e) < 1e-3 and np.max(e) < 2e-2), (r, np.mean(e), np.max(e))
