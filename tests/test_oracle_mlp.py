"""Pins for the FP64 MLP oracle of the learned projection: finite-difference
gradients, the zero-last-layer = copy identity, the feature definition on a
hand-checkable graph, and Adam's first step (|step| = lr per coordinate)."""
import numpy as np

import synth
from oracle import mlp


def rand_params(rng, din, h, dout):
    return (rng.normal(size=(h, din)) * 0.3, rng.normal(size=h) * 0.1,
            rng.normal(size=(dout, h)) * 0.3, rng.normal(size=dout) * 0.1)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    din, h, dout, B = 9, 7, 4, 5
    W1, b1, W2, b2 = rand_params(rng, din, h, dout)
    X, R = rng.normal(size=(B, din)), rng.normal(size=(B, dout))
    L, dW1, db1, dW2, db2 = mlp.loss_and_grads(W1, b1, W2, b2, X, R)
    eps = 1e-6
    for P, G in ((W1, dW1), (b1, db1), (W2, dW2), (b2, db2)):
        flat, gflat = P.reshape(-1), G.reshape(-1)
        for i in rng.choice(flat.size, min(flat.size, 12), replace=False):
            old = flat[i]
            flat[i] = old + eps
            lp = mlp.loss_and_grads(W1, b1, W2, b2, X, R)[0]
            flat[i] = old - eps
            lm = mlp.loss_and_grads(W1, b1, W2, b2, X, R)[0]
            flat[i] = old
            assert abs((lp - lm) / (2 * eps) - gflat[i]) <= 1e-6 * max(1.0, abs(gflat[i]))


def test_zero_last_layer_is_copy_projection():
    rng = np.random.default_rng(1)
    g = synth.rmat_graph(6, 4, 3)
    nc, d = 10, 4
    mp = rng.integers(0, nc, g.n)
    Mc = rng.normal(size=(nc, d))
    X = mlp.features(g.rowptr, g.col, mp, Mc)
    W1, b1, _, _ = rand_params(rng, 2 * d + 1, 6, d)
    Y, _ = mlp.forward(W1, b1, np.zeros((d, 6)), np.zeros(d), X)
    np.testing.assert_array_equal(Mc[mp] + Y, Mc[mp])


def test_features_by_hand():
    # path 0-1-2, map = [0, 1, 1], Mc rows (1,0) and (0,2)
    g = synth.csr_from_edges(3, np.array([0, 1]), np.array([1, 2]), compact=False)
    Mc = np.array([[1.0, 0.0], [0.0, 2.0]])
    X = mlp.features(g.rowptr, g.col, np.array([0, 1, 1]), Mc)
    np.testing.assert_allclose(X[0], [1, 0, np.log(2), 0, 2])            # neighbour 1 -> row 1
    np.testing.assert_allclose(X[1], [0, 2, np.log(3), 0.5, 1])          # mean of rows 0 and 1
    np.testing.assert_allclose(X[2], [0, 2, np.log(2), 0, 2])


def test_adam_first_step_is_lr_sign():
    g = np.array([3.0, -0.5, 1e-3])
    p = np.zeros(3)
    m, v = np.zeros(3), np.zeros(3)
    mlp.adam(p, g, m, v, 1, 0.01)
    np.testing.assert_allclose(p, -0.01 * np.sign(g), rtol=1e-4)
