"""The initial-guess network on the GPU vs the FP64 oracle, its training, and
what it gains over plain Levenberg-Marquardt.

Tolerances for the BF16 tensor-core kernels (8-bit mantissa operands, FP32
accumulation): against the oracle evaluated with the same operands rounded
to bfloat16, element by element within a small multiple of one bfloat16
rounding step (2^-8) of each value's magnitude; against the unrounded FP64
network, raw outputs within 0.05 (standardised units), loss within 2 %,
every layer's gradient within 5 % relative L2 error.
"""
import numpy as np
import pytest

import workloads as W
from oracle import lm, me, mlp
from gpu_common import LINE, T, X, f32, vf  # noqa: F401

pytestmark = pytest.mark.gpu


def _oracle_set(n, seed):
    p = f32(W.training_params(n, seed))
    s = me.synth(p, f32(T), f32(X), LINE).reshape(n, -1)
    obs, w = W.observe(s, p, W.noise(n, 24, seed))
    return p, f32(obs), f32(w)


def _random_blob(seed, obs, params):
    rng = np.random.default_rng(seed)
    weights = [(rng.uniform(-1, 1, (a, b)) * np.sqrt(6.0 / a), rng.normal(0, 0.05, b))
               for a, b in zip(mlp.LAYERS[:-1], mlp.LAYERS[1:])]
    return f32(mlp.pack(weights, mlp.statistics(obs, params)))


def test_init_statistics_match_oracle(vf):
    v, h, torch = vf
    p, obs, w = _oracle_set(4096, 40)
    blob = v.vfisv_nn_init(h, obs.astype(np.float32), p.astype(np.float32), seed=7)
    _, st = mlp.unpack(blob)
    ref = mlp.statistics(obs, p)
    for k in ref:
        np.testing.assert_allclose(st[k], ref[k], rtol=2e-4, atol=1e-6)
    v.vfisv_check(h)  # the device error words stay clear
    lay = mlp.blob_layout()
    W0 = blob[lay["W0"][0]:lay["W0"][0] + 24 * 256]
    assert np.abs(W0).max() <= np.sqrt(6 / 24) and abs(W0.mean()) < 0.02
    assert np.all(blob[lay["b0"][0]:lay["b0"][0] + 256] == 0)


def test_forward_and_gradient_vs_oracle(vf):
    """Loss and gradient of vfisv_nn_grad against the oracle.

    Element by element against the oracle's rounded-operand reading of the
    training kernels (bfloat16 features, weights, activations and output /
    input gradients, exact products, FP64 sums): each entry g_ij = sum_m
    h_mi d_mj may differ by the FP32 accumulation and by the rare operand
    that rounds to the neighbouring bfloat16 value, i.e. by a small multiple
    of 2^-8 of its magnitude sum S_ij = sum_m |h_mi| |d_mj|.  Then, as a
    whole, against the unrounded FP64 backward (raw outputs, loss, per-layer
    relative L2 error of the gradient)."""
    v, h, torch = vf
    p, obs, w = _oracle_set(1000, 41)
    blob = _random_blob(1, obs, p)
    L_b, g_b, y_b, S = mlp.loss_and_grad(blob, obs, p, operand_round=mlp.round_bf16,
                                         want_scale=True)
    loss, g = v.vfisv_nn_grad(h, blob.astype(np.float32), obs.astype(np.float32),
                              p.astype(np.float32))
    g = g.astype(np.float64)
    r = np.abs(g - g_b) / np.maximum(S, 1e-30)
    print(f"\n|g - g_bf16| / S: max {r.max():.3e} p99.9 {np.percentile(r, 99.9):.3e} "
          f"median {np.median(r):.3e}; loss {loss[0]:.6f} vs {L_b:.6f}")
    assert np.median(r) < 2.0 ** -12
    assert np.mean(r <= 2.0 ** -8) >= 0.999
    assert r.max() <= 4 * 2.0 ** -8
    assert abs(loss[0] / L_b - 1) < 1e-3
    # against the exact FP64 network
    L_ref, g_ref, y_ref = mlp.loss_and_grad(blob, obs, p)
    r2 = v.vfisv_nn_infer(h, blob.astype(np.float32), obs.astype(np.float32), LINE, want_raw=True)
    assert np.abs(r2["raw"] - y_ref).max() < 0.05
    assert abs(loss[0] / L_ref - 1) < 2e-2
    lay = mlp.blob_layout()
    for name in ("W0", "b0", "W1", "b1", "W2", "b2", "W3", "b3"):
        o, shp = lay[name]
        n = int(np.prod(shp))
        a, b = g[o:o + n], g_ref[o:o + n]
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert rel < 5e-2, (name, rel)


@pytest.mark.parametrize("n", [1, 128, 1000, 20000])
def test_tensor_core_forward_vs_rounded_operand_oracle(vf, n):
    """The fused tensor-core inference against the oracle forward with every
    layer's operands rounded to bfloat16 (the kernel's operand precision) and
    exact products: what remains is FP32 accumulation order and the rare
    activation that rounds to the neighbouring bfloat16 value.  n spans one
    partial tile, one full tile, several tiles with a ragged tail, and more
    tiles than the persistent grid (several tiles per CTA)."""
    v, h, torch = vf
    rng = np.random.default_rng(43 + n)
    p = f32(W.training_params(n, 43 + n))
    obs = f32(me.synth(p, f32(T), f32(X), LINE).reshape(n, -1)
              * (1.0 + 1e-3 * rng.standard_normal((n, 24))))
    ps, os_, _ = _oracle_set(512, 44)  # standardisation statistics from their own sample
    blob = _random_blob(3, os_, ps)
    weights, st = mlp.unpack(blob)
    y_ref, _ = mlp.forward(weights, mlp.features(obs, st), operand_round=mlp.round_bf16)
    r = v.vfisv_nn_infer(h, blob.astype(np.float32), obs.astype(np.float32), LINE, want_raw=True)
    err = np.abs(r["raw"] - y_ref)
    # most outputs agree to FP32 accumulation order; an activation that lands
    # on the other side of a bfloat16 rounding boundary moves by one bfloat16
    # step (2^-8 relative) and carries that through the later layers
    assert np.median(err) < 1e-5 and err.mean() < 2e-4 and err.max() < 3e-2, \
        (np.median(err), err.mean(), err.max())
    np.testing.assert_array_equal(r["conf"], r["raw"][:, 10])
    v.vfisv_check(h)
    m = mlp.decode(r["raw"].astype(np.float64), obs, st)
    np.testing.assert_allclose(r["init"][:, [0, 3, 5, 6, 7, 8]], m[:, [0, 3, 5, 6, 7, 8]],
                               rtol=2e-5, atol=2e-3)


def test_decoded_guesses_vs_oracle(vf):
    v, h, torch = vf
    p, obs, w = _oracle_set(512, 42)
    blob = _random_blob(2, obs, p)
    r = v.vfisv_nn_infer(h, blob.astype(np.float32), obs.astype(np.float32), LINE, want_raw=True)
    _, st = mlp.unpack(blob)
    # decode the GPU's own raw outputs in FP64: checks the decoding kernel alone
    m = mlp.decode(r["raw"].astype(np.float64), obs, st)
    ok = np.abs(np.cos(np.radians(m[:, 1]))) < 0.999  # away from the arccos poles
    np.testing.assert_allclose(r["init"][:, [0, 3, 4, 5, 6, 7, 8]], m[:, [0, 3, 4, 5, 6, 7, 8]],
                               rtol=2e-5, atol=2e-3)
    np.testing.assert_allclose(r["init"][ok, 1], m[ok, 1], atol=2e-3)
    dpsi = np.abs(np.mod(r["init"][:, 2] - m[:, 2] + 90, 180) - 90)
    assert dpsi.max() < 2e-3


def _gpu_training_set(v, h, torch, n, seed):
    dev = torch.device("cuda:0")
    p = W.training_params(n, seed).astype(np.float32)
    tp = torch.tensor(p, device=dev)
    tf = torch.tensor(T, dtype=torch.float32, device=dev)
    tx = torch.tensor(X, dtype=torch.float32, device=dev)
    s = v.vfisv_synth(h, tp, tf, tx, LINE).reshape(n, 24)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    sig = 1e-3 * (tp[:, 7] + tp[:, 8])[:, None]
    obs = s + sig * torch.randn(n, 24, device=dev, generator=g)
    return tp, obs.contiguous(), tf, tx


def test_training_reduces_loss(vf):
    v, h, torch = vf
    tp, obs, tf, tx = _gpu_training_set(v, h, torch, 65536, 43)
    blob = v.vfisv_nn_init(h, obs, tp, seed=3)
    loss = v.vfisv_nn_train(h, blob, obs, tp, batch=4096, epochs=6, lr0=1e-3, seed=5)
    v.vfisv_check(h)
    l = loss.cpu().numpy()
    assert np.all(np.isfinite(l))
    assert l[-8:].mean() < 0.5 * l[:4].mean(), (l[:4], l[-8:])


def test_network_gain_over_plain_lm(vf):
    """Trained on 1M GPU-synthesised profiles, the network's guesses make the
    inversion of a held-out map converge in fewer iterations, and the mixed
    result (NN + LM, flagged pixels re-inverted plainly) matches or beats
    plain LM's chi2 for nearly every pixel."""
    v, h, torch = vf
    tp, obs, tf, tx = _gpu_training_set(v, h, torch, 1 << 20, W.SEEDS["nn_train"])
    blob = v.vfisv_nn_init(h, obs, tp, seed=11)
    v.vfisv_nn_train(h, blob, obs, tp, batch=8192, epochs=4, lr0=1e-3, seed=12)
    del obs
    n = 16384
    hp, hobs, _, _ = _gpu_training_set(v, h, torch, n, W.SEEDS["nn_heldout"])
    sig = 1e-3 * (hp[:, 7] + hp[:, 8])[:, None]
    wts = (1.0 / (sig * sig)).expand(n, 24).contiguous()
    plain = v.vfisv_invert(h, hobs, wts, tf, tx, LINE)
    mixed = v.vfisv_invert_nn(h, blob, hobs, wts, tf, tx, LINE, chi2_flag=3.0)
    nn_only = v.vfisv_invert(h, hobs, wts, tf, tx, LINE,
                             init=v.vfisv_nn_infer(h, blob, hobs, LINE)["init"],
                             config={"max_iter": 20})
    v.vfisv_check(h)
    c = lambda st: ((st == 0) | (st == 2)).float().mean().item()  # noqa: E731
    it_plain = plain["iters"].float().mean().item()
    it_nn = nn_only["iters"].float().mean().item()
    better = (mixed["chi2"] <= plain["chi2"] * (1 + 1e-3)).float().mean().item()
    print(f"plain: conv {c(plain['status']):.3f} iters {it_plain:.1f}; NN-init: conv "
          f"{c(nn_only['status']):.3f} iters {it_nn:.1f}; mixed conv {c(mixed['status']):.3f} "
          f"flagged {mixed['flagged'].float().mean().item():.3f}; chi2 <= plain: {better:.3f}")
    assert it_nn < 0.7 * it_plain
    assert c(mixed["status"]) >= c(plain["status"])
    assert better >= 0.9


_ORACLE_BLOB = {}


def _oracle_blob():
    """A network trained by the oracle (FP64 Adam) on oracle-synthesised
    profiles, so that no oracle input comes from the CUDA path."""
    if "blob" not in _ORACLE_BLOB:
        tp, tobs, tw = _oracle_set(16384, 46)
        _ORACLE_BLOB["blob"] = f32(mlp.train(tobs, tp, steps=150, batch=1024, lr0=2e-3, seed=3))
    return _ORACLE_BLOB["blob"]


def test_mixed_first_stage_vs_oracle(vf):
    """The network's guess on the GPU (BF16) vs the oracle's FP64 evaluation of
    the same network, and LM from that guess on both sides."""
    v, h, torch = vf
    p, obs, w = _oracle_set(600, 44)
    blob = _oracle_blob()
    weights, st = mlp.unpack(blob)
    y, _ = mlp.forward(weights, mlp.features(obs, st))
    init_ref = mlp.decode(y, obs, st)
    r = v.vfisv_nn_infer(h, blob.astype(np.float32), obs.astype(np.float32), LINE)
    assert np.median(np.abs(r["init"][:, 0] - init_ref[:, 0])) < 30.0
    init = f32(init_ref)
    g = v.vfisv_invert(h, obs.astype(np.float32), w.astype(np.float32), T.astype(np.float32),
                       X.astype(np.float32), LINE, init=init.astype(np.float32),
                       config={"max_iter": 20})
    ref = lm.invert(obs, w, f32(T), f32(X), LINE, init=init, max_iter=20)
    both = np.isin(g["status"], (0, 2)) & np.isin(ref["status"], (0, 2))
    rel = np.abs(g["chi2"][both] / ref["chi2"][both] - 1)
    assert both.mean() > 0.3 and np.mean(rel <= 1e-3) >= 0.98


def test_mixed_pipeline_vs_oracle(vf):
    """vfisv_invert_nn vs the oracle's mixed inversion with the same network
    (trained by the oracle itself, in FP64): flags, and chi2 of pixels
    converged in both."""
    v, h, torch = vf
    blob = _oracle_blob()
    p, obs, w = _oracle_set(600, 47)
    ref = lm.invert_mixed(obs, w, f32(T), f32(X), LINE, blob, nn_cap=20, plain_cap=50,
                          chi2_flag=3.0, flag_unconverged=True)
    g = v.vfisv_invert_nn(h, blob.astype(np.float32), obs.astype(np.float32),
                          w.astype(np.float32), T.astype(np.float32), X.astype(np.float32),
                          LINE, chi2_flag=3.0, flag_unconverged=True)
    assert np.mean(g["flagged"] == ref["flagged"]) >= 0.85
    both = np.isin(g["status"], (0, 2)) & np.isin(ref["status"], (0, 2))
    rel = np.abs(g["chi2"][both] / ref["chi2"][both] - 1)
    assert both.mean() > 0.5 and np.mean(rel <= 1e-3) >= 0.95


def test_confidence_routing_bit_exact(vf):
    """Routing by the confidence output: every routed pixel ends with exactly
    the result of a plain vfisv_invert call (standard guess, cfg_plain), every
    unrouted pixel that is not flagged with exactly the result of LM from the
    network's guess (cfg_nn), and every routed pixel is reported as flagged.
    Two thresholds: half the pixels routed, and none."""
    v, h, torch = vf
    tp, obs, tf, tx = _gpu_training_set(v, h, torch, 3000, 48)
    blob = v.vfisv_nn_init(h, obs, tp, seed=4)
    v.vfisv_nn_train(h, blob, obs, tp, batch=512, epochs=2, lr0=1e-3, seed=6)
    sig = 1e-3 * (tp[:, 7] + tp[:, 8])[:, None]
    wts = (1.0 / (sig * sig)).expand(obs.shape[0], 24).contiguous()
    g = v.vfisv_nn_infer(h, blob, obs, LINE)
    cn, cp = {"max_iter": 25}, {"max_iter": 40}
    plain = v.vfisv_invert(h, obs, wts, tf, tx, LINE, config=cp)
    first = v.vfisv_invert(h, obs, wts, tf, tx, LINE, init=g["init"], config=cn)
    for k in (float(g["conf"].median().item()), float("inf")):
        m = v.vfisv_invert_nn(h, blob, obs, wts, tf, tx, LINE, config_nn=cn, config_plain=cp,
                              chi2_flag=2.5, flag_unconverged=True, conf_route=k)
        v.vfisv_check(h)
        routed = g["conf"] > k
        assert torch.all(m["flagged"][routed] == 1)
        keep = ~routed & (m["flagged"] == 0)
        for key in ("params", "chi2", "status", "cov"):
            assert torch.equal(m[key][routed], plain[key][routed]), key
            assert torch.equal(m[key][keep], first[key][keep]), key
        assert torch.equal(m["iters"][routed], plain["iters"][routed])
        assert torch.equal(m["iters"][keep], first["iters"][keep])
        if k == float("inf"):
            assert not routed.any()
        else:
            assert 0.3 < routed.float().mean().item() < 0.7
