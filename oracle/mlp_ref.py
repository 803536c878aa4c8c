"""FP64 CPU reference of the learned primitive-recovery guess -- TEST
INFRASTRUCTURE ONLY (tests, smoke, benchmark CPU baseline).

The network (not part of the paper; it only provides an initial guess for the
root solve of Sec. 3) maps 10 features of a cell to 4 outputs through two
hidden layers of 64 SiLU units:
    h1 = silu(W1 x + b1), h2 = silu(W2 h1 + b2), y = W3 h2 + b3,
silu(z) = z / (1 + exp(-z)).  Parameters are packed in one vector:
    W1 (64x10, row-major) | b1 (64) | W2 (64x64) | b2 (64) | W3 (4x64) | b3 (4)
(5124 values).  Loss: mean over samples of the squared error summed over the
4 outputs.  The gradient below is plain reverse-mode differentiation of that
definition; the test suite pins it against central finite differences.
"""
from __future__ import annotations

import numpy as np

NIN, NHID, NOUT = 10, 64, 4
SHAPES = [("W1", (NHID, NIN)), ("b1", (NHID,)), ("W2", (NHID, NHID)), ("b2", (NHID,)),
          ("W3", (NOUT, NHID)), ("b3", (NOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(params):
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(params[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def _sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(params, X):
    p = unpack(params)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = z1 * _sigmoid(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = z2 * _sigmoid(z2)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (X, z1, h1, z2, h2)


def loss_and_grad(params, X, Y):
    p = unpack(params)
    y, (X, z1, h1, z2, h2) = forward(params, X)
    n = X.shape[0]
    r = y - np.asarray(Y, dtype=np.float64)
    loss = float(np.sum(r * r) / n)
    dy = 2.0 * r / n
    g = {}
    g["W3"] = dy.T @ h2
    g["b3"] = dy.sum(axis=0)
    dh2 = dy @ p["W3"]
    s2 = _sigmoid(z2)
    dz2 = dh2 * s2 * (1.0 + z2 * (1.0 - s2))
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    s1 = _sigmoid(z1)
    dz1 = dh1 * s1 * (1.0 + z1 * (1.0 - s1))
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return loss, pack(g)


def init_params(seed=0):
    """Seeded initial parameters (uniform +-1/sqrt(fan_in) weights, zero biases)."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, shape in SHAPES:
        if name.startswith("W"):
            lim = 1.0 / np.sqrt(shape[1])
            d[name] = rng.uniform(-lim, lim, shape)
        else:
            d[name] = np.zeros(shape)
    return pack(d)
