"""FP64 CPU oracle of the launch-shape cost model (a 2-layer MLP).

TEST INFRASTRUCTURE ONLY (imported by the tests, never by the library).

The cost model is not in the paper (it serves the launch-shape selection
the library adds).  Its definition, restated here from the textbook:

  parameters, one flat array:  W1 (d x h, row-major: W1[i, j] maps input i
  to hidden unit j), b1 (h), W2 (h x h), b2 (h), w3 (h), b3 (1)
  forward:   h1 = relu(x W1 + b1),  h2 = relu(h1 W2 + b2),  y = h2 . w3 + b3
  loss:      L = (1 / B) sum_b (y_b - t_b)^2  over a batch of B rows of x
  gradient:  back-propagation (chain rule); relu'(0) is taken as 0
  update:    Adam (Kingma and Ba, 2015) with bias correction:
             m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
             p -= lr * (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps)
"""
from __future__ import annotations

import numpy as np


def n_params(d: int, h: int) -> int:
    return d * h + h + h * h + h + h + 1


def unpack(p: np.ndarray, d: int, h: int):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + d * h].reshape(d, h); o += d * h
    b1 = p[o:o + h]; o += h
    W2 = p[o:o + h * h].reshape(h, h); o += h * h
    b2 = p[o:o + h]; o += h
    w3 = p[o:o + h]; o += h
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def forward(p, x, d: int, h: int):
    """y (B,) and the hidden activations (h1, h2)."""
    W1, b1, W2, b2, w3, b3 = unpack(p, d, h)
    x = np.asarray(x, dtype=np.float64).reshape(-1, d)
    h1 = np.maximum(x @ W1 + b1, 0.0)
    h2 = np.maximum(h1 @ W2 + b2, 0.0)
    return h2 @ w3 + b3, h1, h2


def loss(p, x, t, d: int, h: int) -> float:
    y, _, _ = forward(p, x, d, h)
    t = np.asarray(t, dtype=np.float64)
    return float(np.mean((y - t) ** 2))


def loss_and_grad(p, x, t, d: int, h: int):
    """(L, dL/dp) with dL/dp packed like p."""
    W1, b1, W2, b2, w3, b3 = unpack(p, d, h)
    x = np.asarray(x, dtype=np.float64).reshape(-1, d)
    t = np.asarray(t, dtype=np.float64)
    B = x.shape[0]
    y, h1, h2 = forward(p, x, d, h)
    L = float(np.mean((y - t) ** 2))
    dy = 2.0 * (y - t) / B
    dw3 = h2.T @ dy
    db3 = np.sum(dy)
    dh2 = np.outer(dy, w3) * (h2 > 0)
    dW2 = h1.T @ dh2
    db2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2.T) * (h1 > 0)
    dW1 = x.T @ dh1
    db1 = dh1.sum(axis=0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, [db3]])
    return L, g


def adam(p, g, m, v, k: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam step (k = 1 for the first); returns (p, m, v) as new arrays."""
    p, g, m, v = (np.asarray(a, dtype=np.float64) for a in (p, g, m, v))
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** k)
    vh = v / (1.0 - b2 ** k)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def numerical_grad(p, x, t, d: int, h: int, step: float = 1e-6):
    """Central differences of the loss, element by element (slow; tiny
    networks only)."""
    p = np.asarray(p, dtype=np.float64).copy()
    g = np.zeros_like(p)
    for i in range(p.size):
        old = p[i]
        p[i] = old + step
        lp = loss(p, x, t, d, h)
        p[i] = old - step
        lm = loss(p, x, t, d, h)
        p[i] = old
        g[i] = (lp - lm) / (2.0 * step)
    return g
