"""FP64 CPU oracle of the surrogate MLP (test infrastructure only).

Network: x -> (W_l x + b_l, GELU) for the hidden layers -> W_L x + b_L, with
GELU in its tanh form x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))); loss
L = 0.5 mean_rows sum_out (y - t)^2.
Parameters use the padded layout of the CUDA library (per layer W [dout x
din] row-major, then b [dout]); the oracle reads only the real block.  The
backward pass is written out by the chain rule; the tests pin it to central
finite differences of the forward pass.
"""
from __future__ import annotations

import math

import numpy as np


_C = math.sqrt(2.0 / math.pi)


def _gelu(x):
    """GELU in its tanh form: x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3)))."""
    return 0.5 * x * (1.0 + np.tanh(_C * (x + 0.044715 * x ** 3)))


def _gelu_grad(x):
    t = np.tanh(_C * (x + 0.044715 * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * _C * (1.0 + 3 * 0.044715 * x * x)


def pad64(n):
    return (n + 63) // 64 * 64


class MLPOracle:
    def __init__(self, n_in, width, depth, n_out):
        self.n_in, self.width, self.depth, self.n_out = n_in, width, depth, n_out
        self.din = [pad64(n_in)] + [width] * depth
        self.dout = [width] * depth + [pad64(n_out)]
        self.real_in = [n_in] + [width] * depth
        self.real_out = [width] * depth + [n_out]
        self.offsets = []
        off = 0
        for a, b in zip(self.din, self.dout):
            self.offsets.append((off, off + a * b))
            off += a * b + b
        self.nparam = off

    def unpack(self, flat):
        """Real (unpadded) W_l [out x in] and b_l [out] as float64."""
        flat = np.asarray(flat, dtype=np.float64)
        Ws, bs = [], []
        for l, (wo, bo) in enumerate(self.offsets):
            W = flat[wo:wo + self.din[l] * self.dout[l]].reshape(self.dout[l], self.din[l])
            Ws.append(W[:self.real_out[l], :self.real_in[l]].copy())
            bs.append(flat[bo:bo + self.dout[l]][:self.real_out[l]].copy())
        return Ws, bs

    def pack_grad(self, gWs, gbs):
        g = np.zeros(self.nparam)
        for l, (wo, bo) in enumerate(self.offsets):
            G = np.zeros((self.dout[l], self.din[l]))
            G[:self.real_out[l], :self.real_in[l]] = gWs[l]
            g[wo:wo + G.size] = G.ravel()
            g[bo:bo + self.real_out[l]] = gbs[l]
        return g

    def forward(self, flat, x, keep=False):
        Ws, bs = self.unpack(flat)
        h = np.asarray(x, dtype=np.float64)
        pres, acts = [], [h]
        for l in range(len(Ws)):
            z = h @ Ws[l].T + bs[l]
            if l < len(Ws) - 1:
                pres.append(z)
                h = _gelu(z)
                acts.append(h)
            else:
                h = z
        return (h, pres, acts) if keep else h

    def loss(self, flat, x, t):
        y = self.forward(flat, x)
        return 0.5 * np.mean(np.sum((y - t) ** 2, axis=1))

    def grad(self, flat, x, t):
        Ws, bs = self.unpack(flat)
        y, pres, acts = self.forward(flat, x, keep=True)
        M = x.shape[0]
        d = (y - t) / M                       # dL/dy
        gWs, gbs = [None] * len(Ws), [None] * len(Ws)
        for l in range(len(Ws) - 1, -1, -1):
            gWs[l] = d.T @ acts[l]
            gbs[l] = d.sum(axis=0)
            if l > 0:
                d = (d @ Ws[l]) * _gelu_grad(pres[l - 1])
        return 0.5 * np.mean(np.sum((y - t) ** 2, axis=1)), self.pack_grad(gWs, gbs)


def bf16_round(a):
    """Round float32 values to the nearest bfloat16 (ties to even), as FP32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    lower = b & 0xFFFF
    q = b >> 16
    up = (lower > 0x8000) | ((lower == 0x8000) & ((q & 1) == 1))
    q = (q + up.astype(np.uint64)) & 0xFFFF
    return (q << 16).astype(np.uint32).view(np.float32)
