"""Initial-guess network in FP64 (oracle).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

The paper's initialisation module (Sec. 5) uses small back-propagation
networks for B, gamma and v_los.  The network here is the one of the
NN-initialised workload: a multilayer perceptron 24 -> 256 -> 256 -> 256 -> 11
with GELU activations (x * Phi(x), Phi the standard normal CDF) on the hidden
layers and a linear output layer.  This module computes, in FP64:

* forward: h_{l+1} = GELU(h_l W_l + b_l) for the hidden layers, y = h_3 W_3 + b_3;
* loss: L = 1/(N*10) sum (y_o - t_o)^2 over the 10 parameter outputs
        + 1/N sum (y_10 - c)^2, with c = log(mean_o (y_o - t_o)^2 + 1e-4)
        held constant (the confidence output learns the log error);
* backward: dL/dW_l, dL/db_l by the chain rule;
* Adam: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
        w -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps),
  with a cosine learning-rate decay lr_t = lr0 * 0.5 * (1 + cos(pi t / T)).

Weights are stored [fan_in, fan_out] (x @ W).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

LAYERS = (24, 256, 256, 256, 11)
NOUT_PARAM = 10


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    cdf = 0.5 * (1.0 + erf(x / np.sqrt(2.0)))
    pdf = np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)
    return cdf + x * pdf


def forward(weights, x):
    """weights = [(W0,b0),...,(W3,b3)]; returns (y, cache)."""
    h = np.asarray(x, dtype=np.float64)
    cache = []
    nl = len(weights)
    for l, (W, b) in enumerate(weights):
        z = h @ W + b
        cache.append((h, z))
        h = gelu(z) if l < nl - 1 else z
    return h, cache


def confidence_target(y, t):
    """c = log(mean_o (y_o - t_o)^2 + 1e-4), the target of output 10."""
    e = y[:, :NOUT_PARAM] - t
    return np.log((e * e).mean(axis=1) + 1e-4)


def loss_and_grad_output(y, t, c=None):
    """Loss and dL/dy for outputs y [N,11] and parameter targets t [N,10].

    The confidence target c is held constant in the gradient; pass it to
    evaluate the loss at other outputs with the same target."""
    n = y.shape[0]
    e = y[:, :NOUT_PARAM] - t
    if c is None:
        c = confidence_target(y, t)
    ec = y[:, NOUT_PARAM] - c
    L = (e * e).sum() / (n * NOUT_PARAM) + (ec * ec).sum() / n
    dy = np.zeros_like(y)
    dy[:, :NOUT_PARAM] = 2.0 * e / (n * NOUT_PARAM)
    dy[:, NOUT_PARAM] = 2.0 * ec / n
    return L, dy


def backward(weights, cache, dy):
    """Gradients [(dW0,db0),...] from dL/dy and the forward cache."""
    grads = [None] * len(weights)
    d = dy
    for l in range(len(weights) - 1, -1, -1):
        h, z = cache[l]
        if l < len(weights) - 1:
            d = d * gelu_grad(z)
        W, _ = weights[l]
        grads[l] = (h.T @ d, d.sum(axis=0))
        d = d @ W.T
    return grads


def cosine_lr(lr0, step, total):
    return lr0 * 0.5 * (1.0 + np.cos(np.pi * min(step, total) / total))


def adam_step(param, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (param, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mhat = m / (1 - b1 ** step)
    vhat = v / (1 - b2 ** step)
    return param - lr * mhat / (np.sqrt(vhat) + eps), m, v
