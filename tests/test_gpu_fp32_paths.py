"""Euler-forward and backward-in-time runs of the FP32 and cell-index forms
against the FP64 oracle (Sect. 2.1.1: RK4 or Euler-forward; execute with a
negative dt runs backward in time).

The FP32 kernels take their own code paths for both: the Euler step is the
one-stage branch of the step function, and backward time moves the FP32 stage
offset down through the cached snapshot interval.  Tolerance as in the other
FP32 parity tests: equal statuses and step counts, mean position error below
1e-3 cell (depth: local layer thickness), largest below 2e-2 cell.
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


def _global(nz, nt=4, res=2.0, seed=21):
    gf = synth.GlobalField(res_deg=res, nz=nz, nt=nt, seed=seed, kmax=20, period=nt * DAY)
    return gf.spec(materialise=True)


def _dequantised(spec, kind):
    d = np.empty(spec.data.shape)
    for s in range(spec.nt):
        for f in range(spec.data.shape[1]):
            q, sc = O.quantise(spec.data[s, f], kind)
            d[s, f] = O.dequantise(q, kind, sc)
    return d


def _check(g, o, spec, what, periodic=True):
    np.testing.assert_array_equal(g["status"], o["status"], err_msg=what)
    np.testing.assert_array_equal(g["step"], o["step"], err_msg=what)
    np.testing.assert_array_equal(g["time"], o["time"], err_msg=what)
    alive = o["status"] == 0
    assert alive.sum() > 100, what
    e = cell_error(g, o, spec, periodic=periodic)[alive]
    assert np.mean(e) < 1e-3 and np.max(e) < 2e-2, (what, np.mean(e), np.max(e))


def _outputs(g, o, spec, what):
    gk = sorted(k for k in g if not isinstance(k, str))
    ok = sorted(k for k in o if not isinstance(k, str))
    assert len(gk) == len(ok) and len(gk) >= 2, (gk, ok)
    for a, b in zip(gk, ok):
        assert a == b, (a, b)
        gs, os_ = g[a], o[b]
        np.testing.assert_array_equal(gs["status"], os_["status"], err_msg=f"{what} t={b}")
        alive = os_["status"] == 0
        e = cell_error(gs, os_, spec)[alive]
        assert np.mean(e) < 1e-3 and np.max(e) < 2e-2, (what, b, np.mean(e), np.max(e))


@pytest.mark.parametrize("form", ["f32_3d", "f32_2d", "cell_f32", "cell_f16"])
def test_euler_forward_fp32_and_cell(pg, form):
    """Euler-forward (one stage per step) in each FP32 form, 3 days of 30 min
    steps on a time-dependent periodic global field, runtime not a multiple
    of dt (the last step is shortened)."""
    spec = _global(nz=8 if form == "f32_3d" else 1)
    data = _dequantised(spec, 0) if form == "cell_f16" else spec.data
    storage = "f16" if form == "cell_f16" else "f32"
    pos = "cell" if form.startswith("cell") else "f32"
    lon, lat, dep = synth.uniform_particles(4000, 13, (0, 360), (-70, 70), (6.0, 900.0),
                                            dtype=np.float32)
    if form != "f32_3d":
        dep = None
    T = 3 * DAY + 1000.0
    o = oracle_run(oracle_field(spec, data), lon, lat, dep, 0.0, 1800.0, T, scheme="euler")
    fs = pg.FieldSet.from_spec(spec, storage=storage)
    ps = pg.ParticleSet(fs, lon, lat, dep, pos=pos)
    g = gpu_run(ps, pg.Kernel("euler"), T, 1800.0)
    assert g["steps"] == o["steps"]
    _check(g["final"], o["final"], spec, form)
    assert (g["final"]["time"][g["final"]["status"] == 0] == T).all()


@pytest.mark.parametrize("form", ["f32_3d", "cell_f32", "cell_bf16"])
@pytest.mark.parametrize("chunk", [0, 7])
def test_backward_in_time_fp32_and_cell(pg, form, chunk):
    """dt < 0 from 3.5 days back over 2.5 days: stage times cross three
    snapshot times downward, output every 12 h, and (chunk = 7) launches end
    at neither an output nor a snapshot time.  Against the oracle at every
    output time."""
    spec = _global(nz=8 if form == "f32_3d" else 1)
    data = _dequantised(spec, 1) if form == "cell_bf16" else spec.data
    storage = "bf16" if form == "cell_bf16" else "f32"
    pos = "cell" if form.startswith("cell") else "f32"
    lon, lat, dep = synth.uniform_particles(3000, 17, (0, 360), (-70, 70), (6.0, 900.0),
                                            dtype=np.float32)
    if form != "f32_3d":
        dep = None
    t0, T, out = 3.5 * DAY, 2.5 * DAY, 0.5 * DAY
    o = oracle_run(oracle_field(spec, data), lon, lat, dep, t0, -1800.0, T, out)
    fs = pg.FieldSet.from_spec(spec, storage=storage)
    ps = pg.ParticleSet(fs, lon, lat, dep, t0=t0, pos=pos)
    if chunk:
        ps.set_tune(block=128, resort_steps=0, chunk_steps=chunk)
    g = gpu_run(ps, pg.Kernel("rk4"), T, -1800.0, out)
    assert g["steps"] == o["steps"]
    _check(g["final"], o["final"], spec, f"{form} chunk {chunk}")
    assert (g["final"]["time"][g["final"]["status"] == 0] == t0 - T).all()
    _outputs(g, o, spec, f"{form} chunk {chunk}")


@pytest.mark.parametrize("ring", [4, 7, 10])
def test_backward_streamed_equals_resident(pg, ring):
    """Backward in time with snapshots streamed through the ring (four slots:
    one-day launches; seven: launches spanning up to two snapshot times, the
    spare slots prefetching; ten: up to four) equals the resident field bit
    for bit."""
    spec = _global(nz=8, nt=5)
    lon, lat, dep = synth.uniform_particles(2000, 19, (0, 360), (-70, 70), (6.0, 900.0),
                                            dtype=np.float32)
    res = []
    for mode in ("resident", "ptrs"):
        if mode == "resident":
            fs = pg.FieldSet.from_spec(spec, storage="f32")
        else:
            fs = pg.FieldSet(spec.lon, spec.lat, spec.depth, mesh="spherical", periodic_lon=True,
                             nfields=spec.data.shape[1], storage="f32")
            fs.set_times(spec.times, spec.period)
            fs.set_ring(ring)
            fs.stream([spec.data[s] for s in range(spec.nt)])
            assert fs.device_bytes() == ring * 4 * 4 * np.prod(spec.data.shape[2:])
        ps = pg.ParticleSet(fs, lon, lat, dep, t0=4.75 * DAY, pos="f32")
        ps.set_tune(block=128, resort_steps=0, chunk_steps=400)
        res.append(gpu_run(ps, pg.Kernel("rk4"), 4.5 * DAY, -1800.0, 2.25 * DAY))
    for k in ("lon", "lat", "depth", "status", "time", "step"):
        np.testing.assert_array_equal(res[1]["final"][k], res[0]["final"][k], err_msg=k)
