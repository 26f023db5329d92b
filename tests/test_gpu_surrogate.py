"""The flow-map surrogate: features, displacements, training, and the run in
which RK4 checks the network and takes over for rejected particles."""
import numpy as np
import pytest

import synth
from tests.helpers import DAY, cell_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1707_05163_gb300 as pg
    pg.load()
    gf = synth.GlobalField(res_deg=2.0, nz=8, nt=6, seed=41, kmax=20, period=6 * DAY)
    spec = gf.spec(materialise=True)
    fs = pg.FieldSet.from_spec(spec, storage="f32")
    return pg, torch, spec, fs


def _features_numpy(spec, lon, lat, dep, t):
    """The 37 inputs, recomputed in FP64 from the field arrays by indexing."""
    nx, ny, nz = len(spec.lon), len(spec.lat), len(spec.depth)
    out = np.zeros((len(lon), 37))
    for p in range(len(lon)):
        q = np.mod(lon[p] - spec.lon[0], 360.0) + spec.lon[0]
        i = min(int(np.searchsorted(spec.lon, q, "right") - 1), nx - 1)
        hi = spec.lon[i + 1] if i < nx - 1 else spec.lon[0] + 360.0
        xi = (q - spec.lon[i]) / (hi - spec.lon[i])
        j = min(int(np.searchsorted(spec.lat, lat[p], "right") - 1), ny - 2)
        eta = (lat[p] - spec.lat[j]) / (spec.lat[j + 1] - spec.lat[j])
        k = min(int(np.searchsorted(spec.depth, dep[p], "right") - 1), nz - 2)
        zeta = (dep[p] - spec.depth[k]) / (spec.depth[k + 1] - spec.depth[k])
        tt = np.mod(t, spec.period)
        s0 = min(int(tt // (spec.period / spec.nt)), spec.nt - 1)
        s1 = (s0 + 1) % spec.nt
        tau = (tt - spec.times[s0]) / (spec.period / spec.nt)
        out[p, :5] = [xi, eta, lat[p] / 90.0, dep[p] / 1000.0, tt / spec.period]
        c = 5
        for dj in range(-1, 3):
            jj = min(max(j + dj, 0), ny - 1)
            for di in range(-1, 3):
                ii = (i + di) % nx
                for f in range(2):
                    a = spec.data[s0, f, k, jj, ii] * (1 - zeta) + spec.data[s0, f, k + 1, jj, ii] * zeta
                    b = spec.data[s1, f, k, jj, ii] * (1 - zeta) + spec.data[s1, f, k + 1, jj, ii] * zeta
                    out[p, c] = (a + (b - a) * tau) / 0.3
                    c += 1
    return out


def test_features_match_direct_indexing(env):
    pg, torch, spec, fs = env
    lon, lat, dep = synth.uniform_particles(300, 2, (0, 360), (-70, 70), (10.0, 800.0),
                                            dtype=np.float32)
    t0 = 1.3 * DAY
    ps = pg.ParticleSet(fs, lon, lat, dep, t0=t0, pos="f32")
    x = pg.surrogate_features(ps).cpu().numpy()
    ref = _features_numpy(spec, lon, lat, dep, t0)
    np.testing.assert_allclose(x, ref, rtol=0, atol=2e-5)


def test_displacement_apply_roundtrip(env):
    pg, torch, spec, fs = env
    lon, lat, dep = synth.uniform_particles(2000, 3, (0, 360), (-60, 60), (10.0, 800.0),
                                            dtype=np.float32)
    a = pg.ParticleSet(fs, lon, lat, dep, pos="f32")
    b = pg.ParticleSet(fs, lon, lat, dep, pos="f32")
    b.execute(pg.Kernel("rk4"), DAY, 1800.0)
    y = pg.displacement(a, b)
    pg.surrogate_apply(a, y, DAY)
    ga, gb = a.get(), b.get()
    ok = gb["status"] == 0
    assert np.max(cell_error(ga, gb, spec)[ok]) < 1e-3
    assert (ga["time"][ok] == DAY).all()


def test_run_rejecting_everything_is_plain_rk4(env):
    pg, torch, spec, fs = env
    lon, lat, dep = synth.uniform_particles(3000, 4, (0, 360), (-60, 60), (10.0, 800.0),
                                            dtype=np.float32)
    net = pg.MLP(37, 64, 2, 3, seed=3)          # untrained: every check fails
    a = pg.ParticleSet(fs, lon, lat, dep, pos="f32")
    stats = pg.surrogate_run(a, net, pg.Kernel("rk4"), nsteps=6, check_every=3, threshold=0.0)
    ref = pg.ParticleSet(fs, lon, lat, dep, pos="f32")
    ref.execute(pg.Kernel("rk4"), 6 * DAY, 1800.0)
    ga, gr = a.get(), ref.get()
    np.testing.assert_array_equal(ga["status"], gr["status"])
    ok = gr["status"] == 0
    assert np.max(cell_error(ga, gr, spec)[ok]) < 1e-5
    assert stats["rejected"] >= 0.99 * ok.sum() * 2
    assert stats["network_steps"] == 6 * 3000


def test_trained_network_saves_rk4_steps_within_its_threshold(env):
    """What the trained network gains over the method it stands in for, judged
    by RK4 itself: the network explains most of the variance of the 24 h RK4
    displacement, and a surrogate run of 10 days with a loose threshold (half
    a cell) spends less than half the RK4 particle-steps of plain RK4 over the
    same days while its final positions stay within the threshold of plain
    RK4's on average."""
    pg, torch, spec, fs = env
    from paper_1707_05163_gb300 import surrogate as S
    x, y = S.make_segments(fs, 120_000, seed=5, groups=24, period=spec.period)
    xt, yt = S.make_segments(fs, 10_000, seed=6, groups=8, period=spec.period)
    net = pg.MLP(37, 128, 3, 3, seed=1)
    losses = S.train(net, x, y, steps=600, batch=4096, lr=2e-3)
    assert losses[-1] < 0.2 * losses[0]
    pred = net.forward(xt).cpu().numpy()[:, :2]
    yt_ = yt.cpu().numpy()[:, :2]
    r2 = 1.0 - np.sum((pred - yt_) ** 2) / np.sum((yt_ - yt_.mean(axis=0)) ** 2)
    assert r2 > 0.6, r2
    n = 4000
    lon, lat, dep = synth.uniform_particles(n, 21, (0, 360), (-60, 60), (10.0, 400.0),
                                            dtype=np.float32)
    K = pg.Kernel("rk4")
    ref = pg.ParticleSet(fs, lon, lat, dep, pos="f32")
    plain_steps = ref.execute(K, 10 * DAY, 1800.0)
    ps = pg.ParticleSet(fs, lon, lat, dep, pos="f32")
    st = pg.surrogate_run(ps, net, K, nsteps=10, check_every=5, threshold=0.5)
    assert st["rk4_particle_steps"] < 0.5 * plain_steps, (st["rk4_particle_steps"], plain_steps)
    g, r = ps.get(), ref.get()
    ok = (g["status"] == 0) & (r["status"] == 0)
    assert ok.mean() > 0.9
    dlon = (g["lon"] - r["lon"] + 180.0) % 360.0 - 180.0
    e = np.maximum(np.abs(dlon), np.abs(g["lat"] - r["lat"]))[ok] / 2.0   # 2-degree cells
    assert np.mean(e) < 0.5, np.mean(e)


def test_fused_network_step_equals_separate_kernels(env):
    """For the surrogate's network shape (37 features, 4 x 256, 3 outputs) a
    network step is one fused tcgen05 kernel (features gathered on chip, the
    network, the displacement applied); with the layer-by-layer engine it is
    three kernels (features, network, apply).  The two compute the same
    features, products and displacements, so whole surrogate runs -- network
    steps, RK4 checks, rejections, re-integration -- end in the same states
    bit for bit; 30,077 particles (235 row tiles and a ragged one)."""
    pg, torch, spec, fs = env
    net = pg.MLP(37, 256, 4, 3, seed=3)
    lon, lat, dep = synth.uniform_particles(30_077, 12, (0, 360), (-70, 70), (10.0, 800.0),
                                            dtype=np.float32)
    K = pg.Kernel("rk4")
    res = []
    for engine in (1, 2):
        net.set_engine(engine)
        ps = pg.ParticleSet(fs, lon, lat, dep, pos="f32")
        st = pg.surrogate_run(ps, net, K, nsteps=4, check_every=2, threshold=0.2)
        res.append((ps.get(), st))
    (a, sa), (b, sb) = res
    for k in ("lon", "lat", "depth", "time", "step", "status", "id"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    assert sa["rejected"] == sb["rejected"] and sa["checked"] == sb["checked"]
    assert 0 < sa["rejected"] < sa["checked"]          # both branches of the check ran
    assert (a["status"] == 0).mean() > 0.5
