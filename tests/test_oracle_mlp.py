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


def test_blob_layout_matches_header():
    import re, os
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "vfisv.h")).read()
    ntrain = int(re.search(r"VFISV_NN_NTRAIN (\d+)", hdr).group(1))
    nblob = int(re.search(r"VFISV_NN_NBLOB (\d+)", hdr).group(1))
    lay = mlp.blob_layout()
    assert lay["_total"][0] == nblob and lay["in_mean"][0] == ntrain


def test_decode_inverts_targets():
    """decode(standardised targets) recovers the model (psi mod 180)."""
    import workloads as W
    from oracle import me
    p = W.quiet_and_active_params(200, 31)
    x = W.wavelength_grid()
    obs = me.synth(p, W.hmi_filters(x), x, W.FE6173).reshape(200, -1)
    st = mlp.statistics(obs, p)
    t = mlp.targets(p, obs, st)
    y = np.concatenate([t, np.zeros((200, 1))], axis=1)
    m = mlp.decode(y, obs, st)
    np.testing.assert_allclose(m[:, [0, 1, 3, 4, 5, 6, 7, 8]], p[:, [0, 1, 3, 4, 5, 6, 7, 8]],
                               rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(np.mod(m[:, 2] - p[:, 2] + 90, 180) - 90, 0, atol=1e-9)
    f = mlp.features(obs, st)
    np.testing.assert_allclose(f.mean(0), 0, atol=1e-9)
    np.testing.assert_allclose(f.std(0), 1, rtol=1e-9)


def test_blob_gradient_vs_finite_differences():
    rng = np.random.default_rng(5)
    import workloads as W
    p = W.quiet_and_active_params(16, 32)
    obs = rng.normal(0.5, 0.1, (16, 24))
    obs[:, :6] = np.abs(obs[:, :6]) + 0.5
    st = mlp.statistics(obs, p)
    weights = [(rng.normal(0, 0.1, (a, b)), rng.normal(0, 0.05, b))
               for a, b in zip(mlp.LAYERS[:-1], mlp.LAYERS[1:])]
    blob = mlp.pack(weights, st)
    L, g, y = mlp.loss_and_grad(blob, obs, p)
    lay = mlp.blob_layout()
    c0 = mlp.confidence_target(y, mlp.targets(p, obs, st))
    for name, idx in (("W0", 5), ("b1", 3), ("W2", 777), ("W3", 40), ("b3", 10)):
        o = lay[name][0] + idx
        bp, bm = blob.copy(), blob.copy()
        bp[o] += 1e-6
        bm[o] -= 1e-6
        f = lambda b: mlp.loss_and_grad_output(mlp.forward(mlp.unpack(b)[0], mlp.features(obs, st))[0],  # noqa: E731
                                               mlp.targets(p, obs, st), c0)[0]
        fd = (f(bp) - f(bm)) / 2e-6
        assert abs(fd - g[o]) < 1e-6 * max(1.0, abs(fd)), (name, fd, g[o])


def test_round_bf16_ties_and_library():
    # ties go to the even neighbour; anything above a tie goes up
    one = 1.0
    assert mlp.round_bf16(one + 2.0 ** -8) == one                  # tie, 1.0 is even
    assert mlp.round_bf16(one + 3 * 2.0 ** -8) == one + 2.0 ** -6  # tie, rounds up to even
    assert mlp.round_bf16(one + 2.0 ** -8 + 2.0 ** -20) == one + 2.0 ** -7
    assert mlp.round_bf16(-(one + 2.0 ** -8 + 2.0 ** -20)) == -(one + 2.0 ** -7)
    assert mlp.round_bf16(0.0) == 0.0
    assert mlp.round_bf16(3.0 * 2.0 ** 100) == 3.0 * 2.0 ** 100
    # FP32 values against the library's float32 -> bfloat16 conversion
    torch = __import__("pytest").importorskip("torch")
    rng = np.random.default_rng(11)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.round_bf16(x.astype(np.float64)), ref)


def test_forward_with_rounded_operands():
    rng = np.random.default_rng(5)
    net = _net(rng)
    x = rng.normal(size=(7, 5))
    y, _ = mlp.forward(net, x)
    yr, cache = mlp.forward(net, x, operand_round=mlp.round_bf16)
    # the same layers written out with rounded operands
    h = x
    for l, (W, b) in enumerate(net):
        z = mlp.round_bf16(h) @ mlp.round_bf16(W) + b
        h = mlp.gelu(z) if l < len(net) - 1 else z
    np.testing.assert_allclose(yr, h, rtol=0, atol=1e-14)
    # the rounding moves each operand by at most 2^-9 relative: a small change
    assert 0 < np.abs(yr - y).max() < 0.05
    # a single layer whose operands are already on the bfloat16 grid: the
    # rounding is the identity
    W, b = mlp.round_bf16(net[0][0]), net[0][1]
    xg = mlp.round_bf16(x)
    np.testing.assert_array_equal(mlp.forward([(W, b)], xg, operand_round=mlp.round_bf16)[0],
                                  xg @ W + b)


def _grad_case(n=400, seed=41):
    import workloads as W
    from oracle import me
    x = W.wavelength_grid()
    T = W.hmi_filters(x)
    p = W.training_params(n, seed)
    s = me.synth(p, T, x, W.FE6173).reshape(n, -1)
    obs, _ = W.observe(s, p, W.noise(n, 24, seed))
    rng = np.random.default_rng(1)
    weights = [(rng.uniform(-1, 1, (a, b)) * np.sqrt(6.0 / a), rng.normal(0, 0.05, b))
               for a, b in zip(mlp.LAYERS[:-1], mlp.LAYERS[1:])]
    return mlp.pack(weights, mlp.statistics(obs, p)), obs, p


def test_rounded_backward_identity_is_the_exact_backward():
    """With an identity rounding the rounded-operand backward runs every
    rounding site and must reproduce the exact FP64 backward (pinned by
    finite differences above) bit for bit: a misplaced operand, transpose or
    activation derivative on the rounded path would show here."""
    blob, obs, p = _grad_case()
    L0, g0, y0 = mlp.loss_and_grad(blob, obs, p)
    L1, g1, y1, sc = mlp.loss_and_grad(blob, obs, p, operand_round=lambda a: a, want_scale=True)
    assert L0 == L1
    np.testing.assert_array_equal(g0, g1)
    np.testing.assert_array_equal(y0, y1)
    assert np.all(sc >= np.abs(g0) - 1e-15)  # |sum h d| <= sum |h| |d|


def test_bf16_backward_within_rounding_of_exact():
    """Rounding every operand to bfloat16 moves each operand by at most 2^-9
    relative, so each gradient entry moves by a small multiple of 2^-8 of its
    magnitude sum S = sum_m |h_mi| |d_mj| (the multiple grows through the four
    layers, as the rounding of one layer feeds the next): |g_bf16 - g| <=
    8 x 2^-8 x S everywhere, and the bulk far below one 2^-8."""
    blob, obs, p = _grad_case()
    _, g0, _ = mlp.loss_and_grad(blob, obs, p)
    _, gb, _, sc = mlp.loss_and_grad(blob, obs, p, operand_round=mlp.round_bf16, want_scale=True)
    r = np.abs(gb - g0) / np.maximum(sc, 1e-300)
    assert r.max() <= 8 * 2.0 ** -8, r.max()
    assert np.median(r) <= 2.0 ** -8
    assert np.any(gb != g0)  # the rounding does act
