"""FP64 reference of the warm-start MLP and its features.

TEST INFRASTRUCTURE ONLY (imported by the tests and nothing else).

  features of row i: [sum_j r_ij y_j / sum_j r_ij, log(1 + n_i), mean_j r_ij]
  net: y = W3 GELU(W2 GELU(W1 x + b1) + b2) + b3, GELU(z) = z Phi(z)
  loss: mean of (y - t)^2 over rows and outputs; Adam(0.9, 0.999, 1e-8)

Pins (tests/test_oracle_mlp.py): GELU against Phi at known points, the
analytic backward against central finite differences of the forward, and a
hand-computed feature row.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

SQRT1_2 = 1.0 / math.sqrt(2.0)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z * SQRT1_2))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z * SQRT1_2)) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def shapes(i, h, o):
    return [(h, i), (h,), (h, h), (h,), (o, h), (o,)]


def unpack(params, i, h, o):
    out, off = [], 0
    for shp in shapes(i, h, o):
        n = int(np.prod(shp))
        out.append(np.asarray(params[off:off + n], np.float64).reshape(shp))
        off += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(p, np.float64).ravel() for p in parts])


def forward(params, X, i, h, o, weights=None):
    """Forward pass; `weights` optionally replaces W1, W2, W3 in the products
    (e.g. their BF16 rounding) while the biases stay as in params."""
    W1, b1, W2, b2, W3, b3 = unpack(params, i, h, o)
    if weights is not None:
        W1, W2, W3 = weights
    X = np.asarray(X, np.float64)
    z1 = X @ W1.T + b1
    h1 = gelu(z1)
    z2 = h1 @ W2.T + b2
    h2 = gelu(z2)
    y = h2 @ W3.T + b3
    return y, (X, z1, h1, z2, h2)


def loss_and_grad(params, X, T, i, h, o, weights=None):
    W1, b1, W2, b2, W3, b3 = unpack(params, i, h, o)
    if weights is not None:
        W1, W2, W3 = weights
    y, (X, z1, h1, z2, h2) = forward(params, X, i, h, o, weights)
    d = y - np.asarray(T, np.float64)
    loss = float(np.mean(d * d))
    dy = 2.0 * d / d.size
    gW3 = dy.T @ h2
    gb3 = dy.sum(0)
    dz2 = (dy @ W3) * gelu_grad(z2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * gelu_grad(z1)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(0)
    return loss, pack([gW1, gb1, gW2, gb2, gW3, gb3])


def adam(params, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def features(indptr, indices, values, Y):
    n_rows = len(indptr) - 1
    f = Y.shape[1]
    out = np.zeros((n_rows, f + 2))
    for r in range(n_rows):
        lo, hi = indptr[r], indptr[r + 1]
        n = hi - lo
        rv = np.asarray(values[lo:hi], np.float64)
        rs = rv.sum()
        if n > 0 and rs != 0:
            out[r, :f] = (rv[:, None] * Y[indices[lo:hi]].astype(np.float64)).sum(0) / rs
        out[r, f] = math.log1p(n)
        out[r, f + 1] = rs / n if n > 0 else 0.0
    return out
