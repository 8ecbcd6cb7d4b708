"""Float64 CPU oracle of the dataflow-selector MLP (6 -> 64 -> 64 -> 4, ReLU).

TEST INFRASTRUCTURE ONLY (tests/ may import it; the product never does). Plain
numpy: forward pass, masked mean-squared loss and its gradient written out layer
by layer, pinned in tests/test_mlp_oracle.py by central finite differences.
Parameter layout (flat float array): W1[6][64] | b1[64] | W2[64][64] | b2[64] |
W3[64][4] | b3[4], W[i][j] from input i to output j.
"""
from __future__ import annotations

import numpy as np

IN, H, OUT = 6, 64, 4
SIZES = [("W1", IN * H), ("b1", H), ("W2", H * H), ("b2", H), ("W3", H * OUT), ("b3", OUT)]
NP = sum(n for _, n in SIZES)


def unpack(p: np.ndarray) -> dict:
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, n in SIZES:
        out[name] = p[o:o + n]
        o += n
    out["W1"] = out["W1"].reshape(IN, H)
    out["W2"] = out["W2"].reshape(H, H)
    out["W3"] = out["W3"].reshape(H, OUT)
    return out


def forward(p, x):
    w = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ w["W1"] + w["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ w["W2"] + w["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w["W3"] + w["b3"]
    return y, (x, z1, h1, z2, h2)


def loss_and_grad(p, x, t, mask):
    """L = sum(mask (y - t)^2) / sum(mask); returns (L, dL/dp as a flat array)."""
    w = unpack(p)
    y, (x, z1, h1, z2, h2) = forward(p, x)
    mask = np.asarray(mask, dtype=np.float64)
    cnt = max(mask.sum(), 1.0)
    d = y - np.asarray(t, dtype=np.float64)
    L = float((mask * d * d).sum() / cnt)
    dy = mask * 2.0 * d / cnt
    gW3 = h2.T @ dy
    gb3 = dy.sum(0)
    dh2 = (dy @ w["W3"].T) * (z2 > 0)
    gW2 = h1.T @ dh2
    gb2 = dh2.sum(0)
    dh1 = (dh2 @ w["W2"].T) * (z1 > 0)
    gW1 = x.T @ dh1
    gb1 = dh1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return L, g
