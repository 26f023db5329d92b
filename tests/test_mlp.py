"""The surrogate MLP: the FP64 oracle pinned by finite differences, and the
CUDA forward / gradient / training against the oracle.

GPU tolerance: the network runs BF16 weights and BF16 activations between
layers with FP32 accumulation, so each layer carries a relative rounding of
about 2^-8; outputs and gradients are compared against the oracle evaluated on
the same BF16-rounded weights with a relative tolerance of 3e-2 of the
largest entry (4 layers of 2^-8 relative rounding, with margin).
"""
import numpy as np
import pytest

from oracle.mlp_oracle import MLPOracle, bf16_round


def _random_params(o, rng, scale=0.3):
    p = np.zeros(o.nparam)
    for l, (wo, bo) in enumerate(o.offsets):
        W = np.zeros((o.dout[l], o.din[l]))
        W[:o.real_out[l], :o.real_in[l]] = rng.normal(size=(o.real_out[l], o.real_in[l])) * \
            scale / np.sqrt(o.real_in[l])
        p[wo:wo + W.size] = W.ravel()
        p[bo:bo + o.real_out[l]] = rng.normal(size=o.real_out[l]) * 0.1
    return p


def test_oracle_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    o = MLPOracle(5, 64, 2, 3)
    p = _random_params(o, rng, scale=1.0)
    x = rng.normal(size=(7, 5))
    t = rng.normal(size=(7, 3))
    loss, g = o.grad(p, x, t)
    assert abs(loss - o.loss(p, x, t)) < 1e-14
    idx = []
    for l, (wo, bo) in enumerate(o.offsets):
        for _ in range(12):
            idx.append(wo + rng.integers(0, o.real_out[l]) * o.din[l] + rng.integers(0, o.real_in[l]))
        idx.append(bo + rng.integers(0, o.real_out[l]))
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (o.loss(p + e, x, t) - o.loss(p - e, x, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-6 * abs(fd), (i, fd, g[i])
    # padded entries carry no gradient
    mask = np.zeros(o.nparam, bool)
    for l, (wo, bo) in enumerate(o.offsets):
        W = np.zeros((o.dout[l], o.din[l]), bool)
        W[:o.real_out[l], :o.real_in[l]] = True
        mask[wo:wo + W.size] = W.ravel()
        mask[bo:bo + o.real_out[l]] = True
    assert (g[~mask] == 0).all()


def test_gelu_of_oracle_is_the_tanh_form_of_x_phi():
    """The tanh form stays within 1e-3 of x Phi(x) (the Gaussian-CDF GELU),
    is exact at 0, odd part x: GELU(x) - GELU(-x) = x, and its derivative
    matches central differences."""
    from oracle.mlp_oracle import _gelu, _gelu_grad
    from scipy.stats import norm
    x = np.linspace(-6, 6, 1201)
    assert np.max(np.abs(_gelu(x) - x * norm.cdf(x))) < 1e-3
    assert _gelu(np.array([0.0]))[0] == 0.0
    np.testing.assert_allclose(_gelu(x) - _gelu(-x), x, rtol=1e-13, atol=1e-13)
    h = 1e-6
    np.testing.assert_allclose(_gelu_grad(x), (_gelu(x + h) - _gelu(x - h)) / (2 * h),
                               rtol=1e-7, atol=1e-8)


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    v = np.concatenate([rng.normal(size=10000) * 10, [1.00390625, 1.005859375, -2.0 ** -130]])
    v = v.astype(np.float32)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(bf16_round(v), ref)


# ------------------------------------------------------------------ GPU ---

@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1707_05163_gb300 as pg
    pg.load()
    return pg, torch


def _close(a, b, rel=3e-2):
    scale = max(np.max(np.abs(b)), 1e-30)
    assert np.max(np.abs(a - b)) <= rel * scale, (np.max(np.abs(a - b)), scale)


@pytest.mark.gpu
@pytest.mark.parametrize("engine", ["mma.sync", "tcgen05", "tcgen05_layers"])
@pytest.mark.parametrize("shape", [(37, 256, 4, 3), (5, 64, 2, 3), (70, 128, 3, 40)])
def test_forward_and_gradient_against_oracle(gpu, shape, engine):
    """The tensor-core engines against the FP64 oracle: mma.sync; tcgen05,
    whose forward on the surrogate's shape (the first) is the fused
    inference kernel; tcgen05 layer by layer.  The tcgen05 engines run the
    products whose widths are 64 or 256; other widths, as in the third
    shape, take the mma.sync products.  Gradients always run layer by
    layer."""
    pg, torch = gpu
    n_in, width, depth, n_out = shape
    net = pg.MLP(n_in, width, depth, n_out, seed=7)
    net.set_engine({"mma.sync": 0, "tcgen05": 1, "tcgen05_layers": 2}[engine])
    o = MLPOracle(n_in, width, depth, n_out)
    rng = np.random.default_rng(1)
    p = _random_params(o, rng).astype(np.float32)
    net.set_params(p)
    M = 4096 + 96          # several row tiles and a ragged tail
    x = rng.normal(size=(M, n_in)).astype(np.float32)
    t = rng.normal(size=(M, n_out)).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    # oracle on the BF16 weights and BF16-rounded inputs the GPU multiplies
    pw = p.copy()
    for l, (wo, bo) in enumerate(o.offsets):
        pw[wo:bo] = bf16_round(pw[wo:bo])
    xr = bf16_round(x).astype(np.float64)
    y = net.forward(xd).cpu().numpy()
    _close(y, o.forward(pw, xr))
    loss, g = net.grad(xd, td)
    oloss, og = o.grad(pw, xr, t.astype(np.float64))
    assert abs(loss - oloss) <= 3e-2 * abs(oloss)
    for l, (wo, bo) in enumerate(o.offsets):
        _close(g[wo:bo], og[wo:bo])
        _close(g[bo:bo + o.dout[l]], og[bo:bo + o.dout[l]])


@pytest.mark.gpu
def test_training_reduces_loss_on_a_smooth_map(gpu):
    pg, torch = gpu
    rng = np.random.default_rng(5)
    M = 8192
    x = rng.uniform(-1, 1, size=(M, 6)).astype(np.float32)
    t = np.stack([np.sin(2 * x[:, 0]) * x[:, 1], x[:, 2] * x[:, 3], np.cos(x[:, 4] + x[:, 5])],
                 axis=1).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    net = pg.MLP(6, 128, 3, 3, seed=1)
    first = net.train_step(xd, td, 2e-3)
    for _ in range(400):
        last = net.train_step(xd, td, 2e-3)
    assert last < 0.05 * first, (first, last)


@pytest.mark.gpu
@pytest.mark.parametrize("M", [1, 127, 128, 129, 5000, 262151])
def test_tcgen05_forward_matches_mma_sync(gpu, M):
    """The tcgen05 engine (TMEM accumulators) and the mma.sync engine multiply
    the same BF16 operands with FP32 accumulation; they differ only in the
    order of the additions and in the BF16 rounding that follows."""
    pg, torch = gpu
    net = pg.MLP(37, 256, 4, 3, seed=11)
    rng = np.random.default_rng(M)
    x = torch.from_numpy(rng.normal(size=(M, 37)).astype(np.float32)).cuda()
    net.set_engine(False)
    y0 = net.forward(x).cpu().numpy()
    net.set_engine(True)
    y1 = net.forward(x).cpu().numpy()
    y2 = net.forward(x).cpu().numpy()
    np.testing.assert_array_equal(y1, y2)
    _close(y1, y0, rel=1e-2)


@pytest.mark.gpu
@pytest.mark.parametrize("M", [1, 100, 128, 129, 40_000, 300_001])
def test_fused_tcgen05_forward_equals_layer_by_layer(gpu, M):
    """The fused inference kernel (activations kept on chip, weights streamed
    in pieces) issues the same tcgen05 products in the same order and applies
    the same epilogue as the layer-by-layer tcgen05 forward, so the outputs
    are identical; ragged row counts and several tiles per CTA."""
    pg, torch = gpu
    net = pg.MLP(37, 256, 4, 3, seed=13)
    rng = np.random.default_rng(M)
    x = torch.from_numpy(rng.normal(size=(M, 37)).astype(np.float32)).cuda()
    net.set_engine(2)                  # tcgen05, layer by layer
    y_layers = net.forward(x).cpu().numpy()
    net.set_engine(1)                  # tcgen05, fused
    y_fused = net.forward(x).cpu().numpy()
    np.testing.assert_array_equal(y_fused, y_layers)
    # after a training step the packed weights follow the new parameters
    t = torch.from_numpy(rng.normal(size=(4096, 3)).astype(np.float32)).cuda()
    xs = torch.from_numpy(rng.normal(size=(4096, 37)).astype(np.float32)).cuda()
    net.train_step(xs, t, 1e-3)
    y2 = net.forward(x).cpu().numpy()
    net.set_engine(2)
    np.testing.assert_array_equal(y2, net.forward(x).cpu().numpy())
    assert not np.array_equal(y2, y_fused)
