"""Float64 reference of the schedule cost model -- TEST INFRASTRUCTURE ONLY.

Only tests/ may use this module.  It writes out the definitions the CUDA
kernels implement, in float64 numpy, with no shared code:
  h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = W3 h2 + b3
  L  = sum_{b,k} m[b,k] (y[b,k] - t[b,k])^2 / sum m
and the gradient of L by the chain rule (backpropagation).  Pinned in
tests/test_costmodel.py by central finite differences in float64.
"""
import numpy as np

IN, H, OUT = 4, 64, 12


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * IN].reshape(H, IN); o += H * IN
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + OUT * H].reshape(OUT, H); o += OUT * H
    b3 = p[o:o + OUT]; o += OUT
    assert o == p.size
    return W1, b1, W2, b2, W3, b3


def forward(p, x):
    W1, b1, W2, b2, W3, b3 = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    h1 = np.maximum(x @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    y = h2 @ W3.T + b3
    return h1, h2, y


def loss(p, x, t, m):
    _, _, y = forward(p, x)
    return float(np.sum(m * (y - t) ** 2) / np.sum(m))


def grad(p, x, t, m):
    """dL/dp by backpropagation, same layout as p."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    h1, h2, y = forward(p, x)
    dy = 2.0 * m * (y - t) / np.sum(m)
    dW3 = dy.T @ h2
    db3 = dy.sum(0)
    dh2 = (dy @ W3) * (h2 > 0)
    dW2 = dh2.T @ h1
    db2 = dh2.sum(0)
    dh1 = (dh2 @ W2) * (h1 > 0)
    dW1 = dh1.T @ x
    db1 = dh1.sum(0)
    return np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
