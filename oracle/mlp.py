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


def round_bf16(x):
    """Round to the nearest bfloat16 value (8 significant bits, the FP32
    exponent range), ties to even: x = m 2^e with 1/2 <= |m| < 1, and m 2^8
    rounded to an integer.  Values far outside the network's range (FP32
    overflow, subnormals) are not handled."""
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.round(m * 256.0), e - 8)


def forward(weights, x, operand_round=None):
    """weights = [(W0,b0),...,(W3,b3)]; returns (y, cache).

    ``operand_round`` (e.g. ``round_bf16``) is applied to every layer's input
    and weight matrix before the product, which is then formed exactly in
    FP64 -- the arithmetic of a tensor-core layer with rounded operands and a
    wide accumulator (biases and activations unrounded)."""
    h = np.asarray(x, dtype=np.float64)
    cache = []
    nl = len(weights)
    for l, (W, b) in enumerate(weights):
        if operand_round is not None:
            h, W = operand_round(h), operand_round(W)
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


def backward(weights, cache, dy, operand_round=None, want_scale=False):
    """Gradients [(dW0,db0),...] from dL/dy and the forward cache.

    With ``operand_round`` (e.g. ``round_bf16``; the forward cache must come
    from ``forward`` with the same rounding, so its layer inputs are already
    rounded) the arithmetic of tensor-core training kernels with rounded
    operands and a wide accumulator: dL/dy is rounded, each layer's weight
    gradient is the exact product of its rounded input and the rounded
    output gradient, its bias gradient the exact column sum of that rounded
    gradient, and the gradient passed down, (d W^T) * GELU'(z) with W
    rounded, is rounded once more.  ``want_scale`` also returns, per layer,
    sum_m |h_mi| |d_mj| and sum_m |d_mj|: the magnitudes that bound how far
    rounding the operands can move each gradient entry."""
    r = operand_round if operand_round is not None else (lambda a: a)
    nl = len(weights)
    grads = [None] * nl
    scale = [None] * nl
    d = r(dy)
    for l in range(nl - 1, -1, -1):
        h, _ = cache[l]
        grads[l] = (h.T @ d, d.sum(axis=0))
        if want_scale:
            scale[l] = (np.abs(h).T @ np.abs(d), np.abs(d).sum(axis=0))
        if l > 0:
            W, _ = weights[l]
            d = r((d @ r(W).T) * gelu_grad(cache[l - 1][1]))
    return (grads, scale) if want_scale else grads


def cosine_lr(lr0, step, total):
    return lr0 * 0.5 * (1.0 + np.cos(np.pi * min(step, total) / total))


def adam_step(param, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (param, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mhat = m / (1 - b1 ** step)
    vhat = v / (1 - b2 ** step)
    return param - lr * mhat / (np.sqrt(vhat) + eps), m, v


# --- the network's view of a pixel (features, targets, decoding) ----------
# Features: f_j = (obs_j / Ic - in_mean_j) / in_std_j with Ic the largest
# Stokes I sample.  Targets (then standardised by out_mean/out_std):
# [B, cos gamma, sin 2psi, cos 2psi, ln eta0, dlambdaD, a, v, S0/Ic, S1/Ic].

NIN = 24
NTARGET = 10
NFILT = 6


def blob_layout():
    """Offsets of the float32 parameter blob: name -> (offset, shape)."""
    shapes = [("W0", (24, 256)), ("b0", (256,)), ("W1", (256, 256)), ("b1", (256,)),
              ("W2", (256, 256)), ("b2", (256,)), ("W3", (256, 11)), ("b3", (11,)),
              ("in_mean", (24,)), ("in_std", (24,)), ("out_mean", (10,)), ("out_std", (10,))]
    out, off = {}, 0
    for name, shp in shapes:
        out[name] = (off, shp)
        off += int(np.prod(shp))
    out["_total"] = (off, ())
    return out


def unpack(blob):
    """Blob -> (weights [(W, b) x 4], stats dict), FP64 copies."""
    lay = blob_layout()
    b = np.asarray(blob, dtype=np.float64)
    get = lambda k: b[lay[k][0]:lay[k][0] + int(np.prod(lay[k][1]))].reshape(lay[k][1])  # noqa: E731
    weights = [(get(f"W{l}"), get(f"b{l}")) for l in range(4)]
    stats = {k: get(k) for k in ("in_mean", "in_std", "out_mean", "out_std")}
    return weights, stats


def pack(weights, stats):
    lay = blob_layout()
    blob = np.zeros(lay["_total"][0], dtype=np.float64)
    for l, (W, b) in enumerate(weights):
        for k, v in ((f"W{l}", W), (f"b{l}", b)):
            o, shp = lay[k]
            blob[o:o + int(np.prod(shp))] = np.asarray(v).ravel()
    for k, v in stats.items():
        o, shp = lay[k]
        blob[o:o + int(np.prod(shp))] = v
    return blob


def continuum_estimate(obs):
    return np.maximum(obs[:, :NFILT].max(axis=1), 1e-30)


def raw_features(obs):
    return obs / continuum_estimate(obs)[:, None]


def raw_targets(params, ic):
    p = np.asarray(params, dtype=np.float64)
    g = np.radians(p[:, 1])
    ps = np.radians(2.0 * p[:, 2])
    return np.stack([p[:, 0], np.cos(g), np.sin(ps), np.cos(ps), np.log(p[:, 3]), p[:, 4],
                     p[:, 5], p[:, 6], p[:, 7] / ic, p[:, 8] / ic], axis=1)


def statistics(obs, params):
    """Standardisation statistics of a training set (mean, population std)."""
    f = raw_features(obs)
    t = raw_targets(params, continuum_estimate(obs))
    sd = lambda a: np.maximum(a.std(axis=0), 1e-6)  # noqa: E731
    return {"in_mean": f.mean(axis=0), "in_std": sd(f), "out_mean": t.mean(axis=0),
            "out_std": sd(t)}


def features(obs, stats):
    return (raw_features(obs) - stats["in_mean"]) / stats["in_std"]


def targets(params, obs, stats):
    return (raw_targets(params, continuum_estimate(obs)) - stats["out_mean"]) / stats["out_std"]


def decode(y, obs, stats, mu=1.0):
    """Network outputs [N, 11] -> initial models [N, 10] (inverse of targets)."""
    ic = continuum_estimate(obs)
    t = y[:, :NTARGET] * stats["out_std"] + stats["out_mean"]
    m = np.empty((len(y), 10))
    m[:, 0] = np.maximum(t[:, 0], 0.0)
    m[:, 1] = np.degrees(np.arccos(np.clip(t[:, 1], -1.0, 1.0)))
    m[:, 2] = np.mod(0.5 * np.degrees(np.arctan2(t[:, 2], t[:, 3])), 180.0)
    m[:, 3] = np.exp(t[:, 4])
    m[:, 4] = t[:, 5]
    m[:, 5] = t[:, 6]
    m[:, 6] = t[:, 7]
    m[:, 7] = t[:, 8] * ic
    m[:, 8] = t[:, 9] * ic / mu
    m[:, 9] = 1.0
    return m


def loss_and_grad(blob, obs, params, operand_round=None, want_scale=False):
    """FP64 loss and gradient (blob layout, trained part) of one batch; with
    ``operand_round`` the rounded-operand reading of forward and backward;
    ``want_scale`` appends the gradient magnitude scales (blob layout)."""
    weights, stats = unpack(blob)
    y, cache = forward(weights, features(obs, stats), operand_round=operand_round)
    L, dy = loss_and_grad_output(y, targets(params, obs, stats))
    zeros = {k: np.zeros_like(v) for k, v in stats.items()}
    ntrain = blob_layout()["in_mean"][0]
    if want_scale:
        grads, scale = backward(weights, cache, dy, operand_round, want_scale=True)
        sc = pack([(a, b) for a, b in scale], zeros)[:ntrain]
    else:
        grads = backward(weights, cache, dy, operand_round)
    g = pack([(gw, gb) for gw, gb in grads], zeros)[:ntrain]
    return (L, g, y, sc) if want_scale else (L, g, y)


def train(obs, params, steps, batch, lr0=1e-3, seed=0):
    """FP64 Adam with cosine decay on (obs, params) pairs; returns a blob.

    He-uniform weights from a numpy generator, zero biases, statistics of the
    training set; minibatches drawn without replacement per epoch."""
    rng = np.random.default_rng(seed)
    weights = [(rng.uniform(-1, 1, (a, b)) * np.sqrt(6.0 / a), np.zeros(b))
               for a, b in zip(LAYERS[:-1], LAYERS[1:])]
    stats = statistics(obs, params)
    blob = pack(weights, stats)
    ntrain = blob_layout()["in_mean"][0]
    m = np.zeros(ntrain)
    v = np.zeros(ntrain)
    n = len(obs)
    order = rng.permutation(n)
    pos = 0
    for t in range(steps):
        if pos + batch > n:
            order = rng.permutation(n)
            pos = 0
        idx = order[pos:pos + batch]
        pos += batch
        _, g, _ = loss_and_grad(blob, obs[idx], params[idx])
        lr = cosine_lr(lr0, t, steps)
        blob[:ntrain], m, v = adam_step(blob[:ntrain], g, m, v, t + 1, lr)
    return blob
