"""The seeded synthetic inputs follow their stated recipe (no GPU).

The workloads stand in for the paper's OGCM fields and particle releases:
a global 1/4-degree grid with a geometric depth axis, a random k^-3
streamfunction flow (horizontally non-divergent, exactly periodic in time,
0.3 m/s surface rms, W of 1e-4 m/s rms vanishing at the top and bottom
levels), uniform particle boxes rounded to FP32, and 256 batched releases.
"""
import numpy as np

import synth
from synth.fields import EARTH_R

DAY = 86400.0


def test_global_axes_of_the_quarter_degree_grid():
    lon, lat, depth = synth.global_axes(0.25, nz=50)
    assert len(lon) == 1440 and len(lat) == 720 and len(depth) == 50
    np.testing.assert_allclose(np.diff(lon), 0.25, rtol=0, atol=1e-12)
    assert lon[0] == 0.0 and lon[-1] == 359.75
    np.testing.assert_allclose(lat[[0, -1]], [-89.875, 89.875], rtol=0, atol=1e-12)
    np.testing.assert_allclose(depth[[0, -1]], [5.0, 5000.0], rtol=1e-12)
    # geometric: a constant ratio 1000^(1/49) between levels, 38 levels above 1000 m
    np.testing.assert_allclose(depth[1:] / depth[:-1], 1000.0 ** (1.0 / 49.0), rtol=1e-12)
    assert int(np.sum(depth <= 1000.0)) == 38


def _field(**kw):
    args = dict(res_deg=4.0, nz=6, nt=5, seed=3, kmax=12)
    args.update(kw)
    return synth.GlobalField(**args)


def test_global_field_rms_and_profiles():
    gf = _field()
    b = gf.base2d(0)
    assert b.shape == (3, gf.ny, gf.nx)
    np.testing.assert_allclose(np.sqrt(np.mean(b[0] ** 2 + b[1] ** 2)), 0.3, rtol=1e-12)
    np.testing.assert_allclose(np.sqrt(np.mean(b[2] ** 2)), 1e-4, rtol=1e-12)
    np.testing.assert_allclose(gf.prof_uv, np.exp(-gf.depth / 1000.0), rtol=1e-15)
    assert gf.prof_w[0] == 0.0 and gf.prof_w[-1] == 0.0 and (gf.prof_w[1:-1] > 0).all()
    # the stored slab is float32(base x profile)
    sl = gf.slab(0, b)
    assert sl.dtype == np.float32
    np.testing.assert_array_equal(sl[1, 2], (b[1] * gf.prof_uv[2]).astype(np.float32))


def test_global_field_is_horizontally_non_divergent():
    """u = -(1/R) dpsi/dlat and v = (1/(R cos lat)) dpsi/dlon with the same
    difference operators: the discrete divergence d(u)/dlon + d(v cos lat)/dlat
    vanishes up to rounding (the two operators act on different axes and
    commute)."""
    gf = _field(with_w=False, nz=1)
    u, v = gf._uv2d_raw(2)
    dlam = np.deg2rad(360.0 / gf.nx)
    dphi = np.deg2rad(180.0 / gf.ny)
    du = (np.roll(u, -1, axis=1) - np.roll(u, 1, axis=1)) / (2 * dlam)
    dv = np.gradient(v * gf._coslat, dphi, axis=0)
    div = du + dv
    scale = np.max(np.abs(du)) + np.max(np.abs(dv))
    assert np.max(np.abs(div)) < 1e-12 * scale
    assert np.max(np.abs(u)) * EARTH_R > 0.0


def test_global_field_is_periodic_in_time():
    gf = _field()
    later = _field()
    later.times = gf.times + gf.period          # the same snapshots one period later
    for s in (0, 3):
        np.testing.assert_allclose(later.base2d(s), gf.base2d(s), rtol=0,
                                   atol=1e-9 * np.max(np.abs(gf.base2d(s))))
    # and it does change within the period
    assert np.max(np.abs(gf.base2d(1) - gf.base2d(0))) > 1e-3 * np.max(np.abs(gf.base2d(0)))


def test_uniform_particles_rounded_to_fp32_inside_their_box():
    lon, lat, dep = synth.uniform_particles(10000, 2, (0.0, 360.0), (-80.0, 80.0), (5.0, 1000.0),
                                            dtype=np.float32)
    for a, (lo, hi) in ((lon, (0.0, 360.0)), (lat, (-80.0, 80.0)), (dep, (5.0, 1000.0))):
        assert a.dtype == np.float64 and (a >= lo).all() and (a <= hi).all()
        np.testing.assert_array_equal(a, a.astype(np.float32).astype(np.float64))
    # the same seed gives the same particles
    again = synth.uniform_particles(10000, 2, (0.0, 360.0), (-80.0, 80.0), (5.0, 1000.0),
                                    dtype=np.float32)
    np.testing.assert_array_equal(again[0], lon)


def test_batched_releases_follow_the_recipe():
    rels = synth.batch_releases(count=256, seed=4)
    assert len(rels) == 256
    n = np.array([r.n for r in rels])
    dt = np.array([r.dt for r in rels])
    rt = np.array([r.runtime for r in rels])
    kind = np.array([r.kind for r in rels])
    assert n.min() >= 1000 and n.max() <= 2_000_000
    assert int(n.sum()) == 63_280_286
    assert set(dt) <= set(synth.DT_DIVISORS) and all(DAY % d == 0 for d in dt)
    assert all(abs(r - round(r / d) * d) == 0 for r, d in zip(rt, dt))
    assert (rt >= 5 * DAY - dt).all() and (rt <= 90 * DAY + dt).all()
    assert set(kind) == {0, 1, 2} and min(np.bincount(kind)) > 256 / 3 * 0.7
    kh = np.array([r.kh for r in rels if r.kind == 1])
    w = np.array([r.w_sink for r in rels if r.kind == 2]) * DAY
    assert (kh >= 1.0).all() and (kh <= 100.0).all()
    assert (w >= 1.0 - 1e-9).all() and (w <= 100.0 + 1e-9).all()
    assert all(r.kh == 0.0 for r in rels if r.kind != 1)
    assert all(r.w_sink == 0.0 for r in rels if r.kind != 2)
