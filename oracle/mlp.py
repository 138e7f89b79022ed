"""FP64 oracle of the learned coarse-to-fine projection (test infrastructure).

Not in the paper (its only learned projection is MILE's, Sec. 7): a residual
two-layer MLP on per-vertex features, trained by mean squared error on pairs
the method itself produces.

  f(v) = [ M_c[map v] | log(1 + deg v) | mean_{w in Gamma(v)} M_c[map w] ]   (2d+1)
  Z1 = f W1^T + b1,  H = relu(Z1),  Y = H W2^T + b2                       (hidden 256, out d)
  projection:  M_f[v] = M_c[map v] + Y(v)
  loss over a batch of B vertices:  L = (1/B) sum_v || Y(v) - (T(v) - M_c[map v]) ||^2

With W2 = 0 and b2 = 0 the projection is exactly the copy projection.
Plain numpy, every step written out; checked against finite differences in
tests/test_oracle_mlp.py.
"""
from __future__ import annotations

import numpy as np


def features(rowptr, col, mp, Mc):
    """Feature rows of the fine vertices (float64, n x (2d+1))."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    mp = np.asarray(mp, dtype=np.int64)
    Mc = np.asarray(Mc, dtype=np.float64)
    n, d = len(rowptr) - 1, Mc.shape[1]
    deg = np.diff(rowptr)
    X = np.zeros((n, 2 * d + 1))
    X[:, :d] = Mc[mp]
    X[:, d] = np.log1p(deg)
    for v in range(n):
        if deg[v] > 0:
            X[v, d + 1:] = Mc[mp[col[rowptr[v]:rowptr[v + 1]]]].mean(axis=0)
    return X


def forward(W1, b1, W2, b2, X):
    Z1 = X @ W1.T + b1
    H = np.maximum(Z1, 0.0)
    Y = H @ W2.T + b2
    return Y, (X, Z1, H)


def loss_and_grads(W1, b1, W2, b2, X, R):
    """R = residual target (T - copy).  Returns (L, dW1, db1, dW2, db2)."""
    B = X.shape[0]
    Y, (X, Z1, H) = forward(W1, b1, W2, b2, X)
    diff = Y - R
    L = float((diff * diff).sum() / B)
    dY = 2.0 * diff / B
    dW2 = dY.T @ H
    db2 = dY.sum(axis=0)
    dH = dY @ W2
    dZ1 = dH * (Z1 > 0)
    dW1 = dZ1.T @ X
    db1 = dZ1.sum(axis=0)
    return L, dW1, db1, dW2, db2


def adam(param, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) with bias correction; t counts from 1."""
    m[:] = b1 * m + (1 - b1) * grad
    v[:] = b2 * v + (1 - b2) * grad * grad
    mhat = m / (1 - b1 ** t)
    vhat = v / (1 - b2 ** t)
    param -= lr * mhat / (np.sqrt(vhat) + eps)
    return param
