"""FP64 reference of the cost-model MLP (test infrastructure).

Only tests/ and bench.py may use this module; the CUDA library has its own
FP32 kernels for the same network and shares no code with it.

Network (one hidden-layer pair, ReLU), on a batch X of shape (B, F):
    h1 = relu(X W1^T + b1)        W1: (H1, F)
    h2 = relu(h1 W2^T + b2)       W2: (H2, H1)
    y  = h2 w3 + b3               w3: (H2,)
loss = mean over the batch of (y - t)^2, t the standardised log pass time.
Gradients follow from the chain rule written out layer by layer; Adam is the
update of Kingma & Ba (2015) with bias correction.

Flat parameter layout (shared with the CUDA side only as a format, like the
gate records): [W1 (row-major) | b1 | W2 (row-major) | b2 | w3 | b3].
"""
from __future__ import annotations

import numpy as np

F, H1, H2 = 32, 64, 64
SIZES = [("W1", (H1, F)), ("b1", (H1,)), ("W2", (H2, H1)), ("b2", (H2,)), ("w3", (H2,)), ("b3", (1,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    assert p.shape == (NPARAMS,)
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SIZES])


def forward(p, X):
    P = unpack(p)
    X = np.asarray(X, np.float64)
    z1 = X @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ P["w3"] + P["b3"][0]
    return y, (X, z1, h1, z2, h2)


def loss(p, X, t):
    y, _ = forward(p, X)
    return float(np.mean((y - np.asarray(t, np.float64)) ** 2))


def grad(p, X, t):
    """Loss and its gradient with respect to the flat parameters."""
    P = unpack(p)
    y, (X, z1, h1, z2, h2) = forward(p, X)
    t = np.asarray(t, np.float64)
    B = X.shape[0]
    dy = 2.0 * (y - t) / B                      # d loss / d y
    g = {"w3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dz2 = np.outer(dy, P["w3"]) * (z2 > 0)      # through relu
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ P["W2"]) * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return float(np.mean((y - t) ** 2)), pack(g)


def adam(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update; step counts from 1.  Returns new (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
