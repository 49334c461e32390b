"""FP64 CPU reference of the surrogate MLP (test infrastructure only).

Network: x -> standardise -> [Linear -> GELU(erf)] x depth -> Linear(2).
Loss per sample: (p0 - (y0 - ymean)/ystd)^2 + BCE-with-logits(p1, y1),
averaged over the batch.  Plain NumPy forward and reverse-mode backward,
pinned by central finite differences in the tests.  Parameters come as a
list of (W [out][in], b [out]) float64 arrays.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def dgelu(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def bf16(x):
    """Round to bfloat16 (nearest, ties to even) and return float64."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(layers, xs):
    """xs: standardised inputs [n][in0]; returns (zs, hs, out)."""
    h = xs
    zs, hs = [], [h]
    for l, (W, b) in enumerate(layers):
        z = h @ W.T + b
        if l < len(layers) - 1:
            zs.append(z)
            h = gelu(z)
            hs.append(h)
        else:
            return zs, hs, z
    raise ValueError("no layers")


def loss_and_grads(layers, xs, Y, ymean=0.0, ystd=1.0):
    n = xs.shape[0]
    zs, hs, out = forward(layers, xs)
    t = (Y[:, 0] - ymean) / ystd
    d0 = out[:, 0] - t
    z, c = out[:, 1], Y[:, 1]
    loss = np.mean(d0 * d0 + np.maximum(z, 0) - z * c + np.log1p(np.exp(-np.abs(z))))
    g = np.zeros_like(out)
    g[:, 0] = 2.0 * d0 / n
    g[:, 1] = (1.0 / (1.0 + np.exp(-z)) - c) / n
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        grads[l] = (g.T @ hs[l], g.sum(axis=0))
        if l > 0:
            g = (g @ W) * dgelu(zs[l - 1])
    return loss, grads, out
