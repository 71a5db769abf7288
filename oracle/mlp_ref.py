"""FP64 oracle of the learned cost model's network (test infrastructure only).

Network 18 -> 32 -> 32 -> 1 with ReLU, flat parameters
W1[32][18] | b1[32] | W2[32][32] | b2[32] | W3[32] | b3, inputs standardised
with (x - mean) * inv_std, loss L = mean((pred - y)^2).  The gradient is the
chain rule written out layer by layer; Adam is the published update (Kingma
& Ba 2015) with bias correction, beta1 0.9, beta2 0.999, eps 1e-8.  Pinned
by central finite differences and Adam's first-step closed form
(tests/test_mlp_oracle.py).
"""
from __future__ import annotations

import numpy as np

NI, NH = 18, 32
NP = NH * NI + NH + NH * NH + NH + NH + 1


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + NH * NI].reshape(NH, NI); o += NH * NI
    b1 = p[o:o + NH]; o += NH
    W2 = p[o:o + NH * NH].reshape(NH, NH); o += NH * NH
    b2 = p[o:o + NH]; o += NH
    W3 = p[o:o + NH]; o += NH
    b3 = p[o]
    return W1, b1, W2, b2, W3, b3


def normalization(X):
    """Column mean and 1/std (population); constant columns keep scale 1."""
    X = np.asarray(X, dtype=np.float64)
    mean = X.mean(axis=0)
    sd = X.std(axis=0)
    inv = np.where(sd > 1e-6, 1.0 / np.where(sd > 0, sd, 1.0), 1.0)
    return mean, inv


def forward(p, X, mean, inv_std):
    W1, b1, W2, b2, W3, b3 = unpack(p)
    Xn = (np.asarray(X, dtype=np.float64) - mean) * inv_std
    z1 = Xn @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    pred = h2 @ W3 + b3
    return pred, (Xn, z1, h1, z2, h2)


def loss(p, X, y, mean, inv_std):
    pred, _ = forward(p, X, mean, inv_std)
    return float(np.mean((pred - np.asarray(y, dtype=np.float64)) ** 2))


def grad(p, X, y, mean, inv_std):
    """dL/dp by backpropagation, in the flat parameter layout."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    pred, (Xn, z1, h1, z2, h2) = forward(p, X, mean, inv_std)
    y = np.asarray(y, dtype=np.float64)
    dpred = 2.0 * (pred - y) / y.size          # dL/dpred
    gW3 = h2.T @ dpred
    gb3 = dpred.sum()
    dz2 = np.outer(dpred, W3) * (z2 > 0)      # through ReLU
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    gW1 = dz1.T @ Xn
    gb1 = dz1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update at step t (t >= 1); returns (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
