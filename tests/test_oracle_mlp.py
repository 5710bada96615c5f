"""Pins of the FP64 oracle's network: GELU values, backward pass by finite
differences, and one Adam step written from its definition."""
import math

import numpy as np

from oracle import mlp


def _net(rng, layers=(5, 7, 6, 11)):
    return [(rng.normal(0, 0.5, (a, b)), rng.normal(0, 0.1, b)) for a, b in zip(layers[:-1], layers[1:])]


def test_gelu_values():
    # GELU(x) = x Phi(x); Phi(1) = 0.8413447460685429, Phi(-0.5) = 0.3085375387259869
    assert mlp.gelu(np.array(1.0)) == np.float64(0.8413447460685429)
    assert abs(mlp.gelu(np.array(-0.5)) - (-0.5 * 0.3085375387259869)) < 1e-16
    x = np.linspace(-5, 5, 41)
    fd = (mlp.gelu(x + 1e-6) - mlp.gelu(x - 1e-6)) / 2e-6
    np.testing.assert_allclose(mlp.gelu_grad(x), fd, atol=1e-9)


def test_backward_vs_finite_differences():
    rng = np.random.default_rng(3)
    net = _net(rng)
    x = rng.normal(size=(9, 5))
    t = rng.normal(size=(9, 10))

    y, cache = mlp.forward(net, x)
    c0 = mlp.confidence_target(y, t)

    def loss(n):
        # the confidence target is held constant in the gradient
        yy, _ = mlp.forward(n, x)
        return mlp.loss_and_grad_output(yy, t, c0)[0]

    _, dy = mlp.loss_and_grad_output(y, t)
    grads = mlp.backward(net, cache, dy)
    h = 1e-6
    for l, (W, b) in enumerate(net):
        for (i, j) in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1), (1, 2)]:
            Wp = [(w.copy(), bb.copy()) for w, bb in net]
            Wm = [(w.copy(), bb.copy()) for w, bb in net]
            Wp[l][0][i, j] += h
            Wm[l][0][i, j] -= h
            fd = (loss(Wp) - loss(Wm)) / (2 * h)
            assert abs(fd - grads[l][0][i, j]) < 1e-6 * max(1.0, abs(fd)), (l, i, j)
        bp = [(w.copy(), bb.copy()) for w, bb in net]
        bm = [(w.copy(), bb.copy()) for w, bb in net]
        bp[l][1][1] += h
        bm[l][1][1] -= h
        fd = (loss(bp) - loss(bm)) / (2 * h)
        assert abs(fd - grads[l][1][1]) < 1e-6 * max(1.0, abs(fd))


def test_adam_first_step_and_cosine():
    g = np.array([0.3, -2.0, 1e-3])
    p = np.array([1.0, 1.0, 1.0])
    p1, m, v = mlp.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=1e-3)
    # bias-corrected first step moves every weight by lr * sign(g) (|g| >> eps)
    np.testing.assert_allclose(p1, p - 1e-3 * np.sign(g) * np.abs(g) / (np.abs(g) + 1e-8), rtol=1e-12)
    assert mlp.cosine_lr(1e-3, 0, 100) == 1e-3
    assert abs(mlp.cosine_lr(1e-3, 50, 100) - 5e-4) < 1e-15
    assert mlp.cosine_lr(1e-3, 100, 100) == 0.0
    assert math.isclose(mlp.cosine_lr(1e-3, 25, 100), 1e-3 * 0.5 * (1 + math.cos(math.pi / 4)))
