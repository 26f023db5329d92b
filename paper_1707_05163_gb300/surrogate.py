"""Training data and training loop of the flow-map surrogate (orchestration of
library calls; features, RK4 segments, displacements and every network
product run in the CUDA library)."""
from __future__ import annotations

import numpy as np

from .api import MLP, Kernel, ParticleSet, displacement, surrogate_features


def make_segments(fieldset, n, seed, horizon=86400.0, dt=1800.0, groups=60, period=None,
                  lat_range=(-80.0, 80.0), depth_range=(5.0, 1000.0)):
    """n RK4 segments of `horizon` seconds from random starts at `groups`
    start times spread over the field's period: returns CUDA tensors
    (features [m x 37], displacement targets [m x 3]) of the m segments whose
    particle stayed in the domain."""
    import torch
    rng = np.random.default_rng(seed)
    per = groups and (n + groups - 1) // groups
    period = period if period is not None else 30 * 86400.0
    xs, ys = [], []
    k = Kernel("rk4")
    done = 0
    for g in range(groups):
        m = min(per, n - done)
        if m <= 0:
            break
        lon = rng.uniform(0.0, 360.0, m).astype(np.float32).astype(np.float64)
        lat = rng.uniform(*lat_range, m).astype(np.float32).astype(np.float64)
        dep = rng.uniform(*depth_range, m).astype(np.float32).astype(np.float64)
        t0 = (g + rng.uniform()) * period / groups
        a = ParticleSet(fieldset, lon, lat, dep, t0=t0, pos="f32")
        b = ParticleSet(fieldset, lon, lat, dep, t0=t0, pos="f32")
        x = surrogate_features(a)
        b.execute(k, horizon, dt)
        y = displacement(a, b)
        st = torch.from_numpy(b.get(sort_by_id=False)["status"]).cuda()
        keep = st == 0
        xs.append(x[keep])
        ys.append(y[keep])
        a.destroy()
        b.destroy()
        done += m
    return torch.cat(xs), torch.cat(ys)


def train(net: MLP, x, y, steps, batch=8192, lr=1e-3, lr_end=1e-5, seed=0, log_every=0):
    """Adam steps on random batches (cosine learning-rate decay); returns the
    list of batch losses."""
    import torch
    gen = torch.Generator(device=x.device)
    gen.manual_seed(seed)
    n = x.shape[0]
    losses = []
    for s in range(steps):
        idx = torch.randint(0, n, (batch,), device=x.device, generator=gen)
        xb = x.index_select(0, idx).contiguous()
        yb = y.index_select(0, idx).contiguous()
        frac = s / max(steps - 1, 1)
        rate = lr_end + 0.5 * (lr - lr_end) * (1.0 + np.cos(np.pi * frac))
        losses.append(net.train_step(xb, yb, rate))
        if log_every and s % log_every == 0:
            print(f"step {s} loss {losses[-1]:.5f}", flush=True)
    return losses
