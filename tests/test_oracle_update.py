"""Pins for UPDATEEMBED (Alg. 1) and the NCE loss (Sec. 2).

- a hand-worked example with exact dyadic values (tests/golden/updateembed_hand.txt)
- central finite differences of the per-sample negative log-likelihood
- the closed form of the sample row after the literal two-line update
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "updateembed_hand.txt")


def test_hand_example(orc):
    rows = np.loadtxt(GOLDEN)
    for b, mv0, mv1, mu0, mu1, lr, ev0, ev1, eu0, eu1 in rows:
        mv, mu, x = orc.update_embed([mv0, mv1], [mu0, mu1], int(b), lr)
        assert x == 0.0
        assert list(mv) == [ev0, ev1]
        assert list(mu) == [eu0, eu1]


def _fd_grad(f, x, h=1e-6):
    g = np.zeros_like(x)
    for i in range(len(x)):
        e = np.zeros_like(x)
        e[i] = h
        g[i] = (f(x + e) - f(x - e)) / (2 * h)
    return g


@pytest.mark.parametrize("b", [0, 1])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_source_step_is_gradient_descent(orc, b, seed):
    rng = np.random.default_rng(seed)
    d, lr = 16, 0.07
    mv = rng.normal(size=d) * 0.4
    mu = rng.normal(size=d) * 0.4
    loss_v = lambda z: orc.sample_loss(float(z @ mu), b)
    grad_v = _fd_grad(loss_v, mv)
    mv1, mu1, x = orc.update_embed(mv, mu, b, lr)
    np.testing.assert_allclose(mv1 - mv, -lr * grad_v, rtol=1e-6, atol=1e-10)
    # closed form of the literal second line: M[u]' = (1 + s^2) M[u] + s M[v]
    s = float(((mv1 - mv) @ mu) / (mu @ mu))
    np.testing.assert_allclose(mu1, (1 + s * s) * mu + s * mv, rtol=1e-12, atol=1e-14)
    # and the sample step is also descent along its own gradient at the old point,
    # up to the second-order term s^2 M[u]
    loss_u = lambda z: orc.sample_loss(float(mv @ z), b)
    grad_u = _fd_grad(loss_u, mu)
    np.testing.assert_allclose(mu1 - mu - s * s * mu, -lr * grad_u, rtol=1e-6, atol=1e-10)


def test_loss_identities(orc):
    for x in [-40.0, -3.0, -1e-3, 0.0, 0.5, 7.0, 40.0]:
        # softplus(-x) - softplus(x) = -x
        assert abs(orc.sample_loss(x, 1) - orc.sample_loss(x, 0) + x) < 1e-12 * max(1, abs(x))
    assert abs(orc.sample_loss(0.0, 1) - np.log(2)) < 1e-15
    # no overflow for large |x|
    assert orc.sample_loss(800.0, 0) == pytest.approx(800.0)
    assert orc.sample_loss(800.0, 1) == pytest.approx(0.0, abs=1e-300)
    # derivative of -log sigma(x) is sigma(x) - 1
    for x in [-2.0, 0.3, 1.7]:
        fd = (orc.sample_loss(x + 1e-6, 1) - orc.sample_loss(x - 1e-6, 1)) / 2e-6
        assert fd == pytest.approx(1 / (1 + np.exp(-x)) - 1, rel=1e-6)


def test_epoch_lr_schedule(orc):
    lr = 0.045
    assert orc.epoch_lr(lr, 1e-4, 0, 10) == lr
    assert orc.epoch_lr(lr, 1e-4, 5, 10) == pytest.approx(lr * 0.5)
    assert orc.epoch_lr(lr, 1e-4, 9, 10) == pytest.approx(lr * 0.1)
    # floor binds when 1 - j/e_i falls below it
    assert orc.epoch_lr(lr, 1e-4, 19999, 20000) == pytest.approx(lr * 1e-4)
    assert orc.epoch_lr(lr, 1e-4, 20000, 20000) == pytest.approx(lr * 1e-4)
