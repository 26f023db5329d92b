"""Failure handling without a GPU fault: every device allocation of the
library is made to fail through the library's allocation limit (a host-side
hook), and each call must return PG_ERR_NOMEM and leave its objects as they
were (the error conventions of the C ABI; the paper's recovery kernels,
Sect. 2.1.2, cover particle errors, these cover the library's own).  Plus
quantised storage of fields with NaN nodes (land): the scale ignores NaN,
as the oracle's does; and the bounded device wait of the tcgen05 kernels
running out on a barrier nothing completes."""
import numpy as np
import pytest

import oracle as O
import synth
from tests.helpers import DAY, gpu_run, oracle_field, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1707_05163_gb300 as pg
    pg.load()
    return pg


class _Limit:
    """Allow `extra` more bytes of library allocations inside the block."""

    def __init__(self, lib, extra):
        self.lib, self.extra = lib, extra

    def __enter__(self):
        assert self.lib.pg_debug_set_alloc_limit(self.extra) == 0

    def __exit__(self, *a):
        self.lib.pg_debug_set_alloc_limit(-1)


def _nomem(pg, fn):
    with pytest.raises(pg.PGError) as e:
        fn()
    assert e.value.code == -7, e.value


def test_allocation_failures_leave_objects_unchanged(pg):
    lib = pg.load()
    gf = synth.GlobalField(res_deg=4.0, nz=6, nt=3, seed=3, kmax=10, period=3 * DAY)
    spec = gf.spec(materialise=True)
    # field set creation
    with _Limit(lib, 0):
        _nomem(pg, lambda: pg.FieldSet(spec.lon, spec.lat, spec.depth, mesh="spherical",
                                       periodic_lon=True, nfields=3, storage="f32"))
    fs = pg.FieldSet(spec.lon, spec.lat, spec.depth, mesh="spherical", periodic_lon=True,
                     nfields=3, storage="f32")
    fs.set_times(spec.times, spec.period)
    # new times: refused, the old ones stay
    with _Limit(lib, 0):
        _nomem(pg, lambda: fs.set_times(np.arange(5) * DAY, 5 * DAY))
    for s in range(2):
        fs.load_snapshot(s, spec.data[s])
    # a snapshot that does not fit: refused, not loaded
    with _Limit(lib, 0):
        _nomem(pg, lambda: fs.load_snapshot(2, spec.data[2]))
    lon, lat, dep = synth.uniform_particles(1000, 4, (0, 360), (-60, 60), (6.0, 500.0),
                                            dtype=np.float32)
    ps = pg.ParticleSet(fs, lon, lat, dep, pos="f32")
    with pytest.raises(pg.PGError) as e:          # snapshot 2 missing
        ps.execute(pg.Kernel("rk4"), DAY, 1800.0)
    assert e.value.code == -3
    fs.load_snapshot(2, spec.data[2])
    # particle-set creation and growth
    with _Limit(lib, 0):
        _nomem(pg, lambda: pg.ParticleSet(fs, lon, lat, dep, pos="f32"))
    before = ps.get()
    with _Limit(lib, 0):
        _nomem(pg, lambda: ps.add(lon, lat, dep))
    after = ps.get()
    assert len(ps) == 1000
    for k in before:
        np.testing.assert_array_equal(before[k], after[k])
    # an execute that needs re-sort scratch: refused before any step
    ps.set_tune(block=128, resort_steps=10, chunk_steps=10)
    with _Limit(lib, 0):
        _nomem(pg, lambda: ps.execute(pg.Kernel("rk4"), DAY, 1800.0))
    after = ps.get()
    for k in before:
        np.testing.assert_array_equal(before[k], after[k], err_msg=k)
    # the streamed ring that does not fit: refused, the field stays resident
    with _Limit(lib, 0):
        _nomem(pg, lambda: fs.stream([spec.data[s] for s in range(spec.nt)]))
    ref = pg.ParticleSet(fs, lon, lat, dep, pos="f32")
    ref.execute(pg.Kernel("rk4"), DAY, 1800.0)
    ps.set_tune(block=128, resort_steps=0, chunk_steps=64)
    ps.execute(pg.Kernel("rk4"), DAY, 1800.0)
    a, b = ps.get(), ref.get()
    for k in ("lon", "lat", "depth", "status", "time"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    # the MLP's workspace
    net = pg.MLP(37, 256, 4, 3, seed=1)
    import torch
    x = torch.zeros((4096, 37), dtype=torch.float32, device="cuda")
    with _Limit(lib, 0):
        _nomem(pg, lambda: net.forward(x))
    assert net.forward(x).shape == (4096, 3)


@pytest.mark.parametrize("storage,kind", [("f16", 0), ("bf16", 1)])
def test_quantised_field_with_nan_nodes(pg, storage, kind):
    """NaN nodes (land) in a quantised field: the per-(field, snapshot) scale
    is the maximum of the finite |values| (NaN ignored, as in the oracle),
    codes of NaN nodes stay NaN, and particles reaching a cell that touches
    them are deleted with PG_NAN; a plane that is NaN everywhere gets the
    scale 1.  Statuses equal the oracle's on the dequantised field."""
    gf = synth.GlobalField(res_deg=2.0, nz=1, nt=3, seed=8, kmax=20, period=3 * DAY)
    spec = gf.spec(materialise=True)
    data = spec.data.astype(np.float32).copy()
    rng = np.random.default_rng(2)
    for _ in range(40):
        i, j = rng.integers(0, spec.data.shape[-1] - 3), rng.integers(5, spec.data.shape[-2] - 8)
        data[:, :, 0, j:j + 3, i:i + 3] = np.nan
    data[2, 1] = np.nan                       # V of snapshot 2 is all land
    spec.data = data
    fs = pg.FieldSet.from_spec(spec, storage=storage)
    dq = np.empty(data.shape)
    for s in range(spec.nt):
        for f in range(2):
            q, sc = O.quantise(data[s, f], kind)
            assert fs.scale(s, f) == sc and np.isfinite(sc)
            dq[s, f] = O.dequantise(q, kind, sc)
    assert fs.scale(2, 1) == 1.0
    lon, lat, _ = synth.uniform_particles(4000, 12, (0, 360), (-70, 70), dtype=np.float32)
    # 0.9 days: stage times stay between snapshots 0 and 1
    o = oracle_run(oracle_field(spec, dq), lon, lat, None, 0.0, 1800.0, 0.9 * DAY)
    g = gpu_run(pg.ParticleSet(fs, lon, lat, pos="f32"), pg.Kernel("rk4"), 0.9 * DAY, 1800.0)
    st = o["final"]["status"]
    assert (st == 3).sum() > 100
    assert np.mean(g["final"]["status"] == st) > 0.99
    assert (g["final"]["status"][st == 3] == 3).mean() > 0.99


def test_bounded_wait_gives_up_and_reports_timeout(pg):
    """The bounded mbarrier wait of the tcgen05 kernels, run on a barrier
    phase that nothing completes (no copy or product in flight), gives up
    after its poll limit; the kernel records it, the call returns
    PG_ERR_TIMEOUT with its message, and the context stays usable: the fused
    tcgen05 forward runs afterwards and matches the layer-by-layer one."""
    import torch
    lib = pg.load()
    for polls in (1, 1000, 100_000):
        assert lib.pg_debug_bounded_wait(polls, None) == -6
        assert b"gave up" in lib.pg_last_error()
    assert lib.pg_debug_bounded_wait(0, None) == -1          # argument checked
    net = pg.MLP(37, 256, 4, 3, seed=2)
    x = torch.randn(1000, 37, device="cuda")
    net.set_engine(1)
    y1 = net.forward(x).cpu().numpy()
    net.set_engine(2)
    y2 = net.forward(x).cpu().numpy()
    assert np.isfinite(y1).all()
    np.testing.assert_array_equal(y1, y2)
