"""fp64 reference of the variant-selector MLP -- TEST INFRASTRUCTURE ONLY.

A 16-64-64-4 network with ReLU hidden layers: h1 = relu(x W1 + b1),
h2 = relu(h1 W2 + b2), y = h2 W3 + b3.  Loss = sum(mask * (y - t)^2) /
max(sum(mask), 1).  Parameters are one flat vector in the order
W1[16][64], b1[64], W2[64][64], b2[64], W3[64][4], b3[4] (5508 values).
Adam: beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias-corrected.

Parity status: pinned by finite differences of the loss and by closed-form
cases (zero hidden weights, a hand-computed tiny network) in tests.
"""
from __future__ import annotations

import numpy as np

F_IN, F_H, F_OUT = 16, 64, 4
SHAPES = [("W1", (F_IN, F_H)), ("b1", (F_H,)), ("W2", (F_H, F_H)), ("b2", (F_H,)),
          ("W3", (F_H, F_OUT)), ("b3", (F_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = w[o:o + size].reshape(shape)
        o += size
    return out


def pack(p) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def forward(w, x):
    """Returns (y, cache) for a batch x of shape [B, 16]."""
    p = unpack(w)
    x = np.asarray(x, dtype=np.float64)
    a1 = x @ p["W1"] + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ p["W3"] + p["b3"]
    return y, (x, a1, h1, a2, h2)


def loss(w, x, t, mask) -> float:
    y, _ = forward(w, x)
    m = np.asarray(mask, dtype=np.float64)
    return float((m * (y - t) ** 2).sum() / max(m.sum(), 1.0))


def grad(w, x, t, mask):
    """Analytic gradient of loss() by the chain rule, layer by layer."""
    p = unpack(w)
    y, (x, a1, h1, a2, h2) = forward(w, x)
    m = np.asarray(mask, dtype=np.float64)
    dy = 2.0 * m * (y - t) / max(m.sum(), 1.0)
    g = {"W3": h2.T @ dy, "b3": dy.sum(0)}
    dh2 = (dy @ p["W3"].T) * (a2 > 0)
    g["W2"] = h1.T @ dh2
    g["b2"] = dh2.sum(0)
    dh1 = (dh2 @ p["W2"].T) * (a1 > 0)
    g["W1"] = x.T @ dh1
    g["b1"] = dh1.sum(0)
    return pack(g)


def adam_step(w, m, v, g, step: int, lr: float):
    b1, b2, eps = 0.9, 0.999, 1e-8
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
