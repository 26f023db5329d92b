"""The allocation-free moments call agrees with pg_pset_moments.

pg_moments_f64_noalloc serves callers that must not allocate device memory
while they run (all device memory owned by their own allocator, or loops
where cudaMalloc/cudaFree round trips and cudaFree's device-wide
synchronisation are not affordable).  It keeps its partial sums in a fixed
device array of the library instead.  This test calls it through the C ABI
twice in a row, on two different particle states, and compares each result
with the allocating entry point on the same particles.  It lives in a file
that pytest collects last, so a run stopping at the first failure has already
run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_moments_match_pset_moments_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1707_05163_gb300 as pg
    lib = pg.load()
    dev = torch.device("cuda", 0)
    spec = synth.stommel_gyre(n=201)
    fs = pg.FieldSet.from_spec(spec, storage="f64")
    n = 1_000_003                      # several blocks and a ragged tail
    rng = np.random.default_rng(17)
    lon = torch.from_numpy(rng.uniform(5e4, 9.5e5, n)).to(dev)
    lat = torch.from_numpy(rng.uniform(5e4, 9.5e5, n)).to(dev)
    ps = pg.ParticleSet(fs, lon, lat, pos="f64")
    out = torch.empty(7, dtype=torch.float64, device=dev)

    def noalloc(x, y, z, status, count):
        out.fill_(-1.0)
        r = lib.pg_moments_f64_noalloc(x.data_ptr(), y.data_ptr(),
                                       z.data_ptr() if z is not None else None,
                                       status.data_ptr() if status is not None else None,
                                       count, out.data_ptr(), None)
        assert r == 0, lib.pg_last_error()
        torch.cuda.synchronize()
        return out.cpu().numpy().copy()

    # call 1: the particles as created (all alive, depth zero)
    ref1 = ps.moments()
    got1 = noalloc(lon, lat, None, None, n)
    assert got1[0] == ref1[0] == n
    np.testing.assert_allclose(got1, ref1, rtol=1e-12, atol=0)

    # call 2: after advecting for 40 days some particles have left the domain
    ps.execute(pg.Kernel("rk4"), 40 * 86400.0, 3600.0)
    x = torch.empty(n, dtype=torch.float64, device=dev)
    y = torch.empty(n, dtype=torch.float64, device=dev)
    z = torch.empty(n, dtype=torch.float64, device=dev)
    st = torch.empty(n, dtype=torch.uint8, device=dev)
    ps.get_into(lon=x, lat=y, depth=z, status=st)
    ref2 = ps.moments()
    # no library allocation may happen inside the call: every allocation of
    # the library fails while the limit is zero
    assert lib.pg_debug_set_alloc_limit(0) == 0
    try:
        got2 = noalloc(x, y, z, st, n)
    finally:
        lib.pg_debug_set_alloc_limit(-1)
    assert got2[0] == ref2[0] == int((st == 0).sum())
    np.testing.assert_allclose(got2, ref2, rtol=1e-12, atol=0)
    assert not np.allclose(got1, got2)

    # beyond the fixed scratch: rejected before any work, output untouched
    out.fill_(-1.0)
    r = lib.pg_moments_f64_noalloc(x.data_ptr(), y.data_ptr(), None, None, (1 << 28) + 1,
                                   out.data_ptr(), None)
    assert r == -1 and b"limit" in lib.pg_last_error()
    torch.cuda.synchronize()
    assert (out.cpu().numpy() == -1.0).all()
