"""GPU Levenberg-Marquardt inversion vs the FP64 oracle on the same inputs.

Parity criteria (the inversion is an iteration run in FP32/FP64 on the GPU
and FP64 in the oracle, so trajectories can part where a trial's chi2 ties
within FP32 rounding; the criteria compare what is unique):
* pixels converged in both (status CONVERGED or STALLED): chi2 within 1e-3
  relative for >= 98 % of them;
* among those, the well-determined ones (B_oracle >= 100 G and oracle
  sigma_gamma, sigma_psi < 5 deg from its covariance): |dB| <= 1 G,
  |dgamma| <= 0.05 deg, |dpsi mod 180| <= 0.05 deg for >= 98 %;
* pixels whose GPU and oracle iteration counts agree follow the same
  trajectory: for them chi2 agrees within 1e-3 relative for all, except
  where the oracle itself lands elsewhere when its inputs are nudged by
  1e-7 (then the equal count is a coincidence).
"""
import numpy as np
import pytest

import workloads as W
from oracle import lm, me
from gpu_common import LINE, T, X, f32, vf  # noqa: F401

pytestmark = pytest.mark.gpu
CONV = (0, 2)


def _case(n, seed, noise=True, scale=None):
    p = f32(W.quiet_and_active_params(n, seed))
    if scale is not None:
        p = f32(scale(p))
    s = me.synth(p, f32(T), f32(X), LINE).reshape(n, -1)
    nz = W.noise(n, 24, seed) if noise else np.zeros((n, 24))
    obs, w = W.observe(s, p, nz)
    return p, f32(obs), f32(w)


def _gpu(v, h, torch, obs, w, init=None, cfg=None, host=False):
    if host:
        r = v.vfisv_invert(h, obs.astype(np.float32), w.astype(np.float32), T.astype(np.float32),
                           X.astype(np.float32), LINE,
                           init=None if init is None else init.astype(np.float32), config=cfg)
        return r
    t = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda:0")  # noqa: E731
    r = v.vfisv_invert(h, t(obs), t(w), t(T), t(X), LINE, init=None if init is None else t(init),
                       config=cfg)
    v.vfisv_check(h)
    return {k: (x.cpu().numpy() if x is not None else None) for k, x in r.items()}


def _compare(g, o):
    both = np.isin(g["status"], CONV) & np.isin(o["status"], CONV)
    rel = np.abs(g["chi2"] / np.where(o["chi2"] > 0, o["chi2"], 1) - 1)
    out = {"both": both, "rel": rel}
    sg = np.sqrt(np.maximum(o["cov"][:, 1, 1], 0))
    sp = np.sqrt(np.maximum(o["cov"][:, 2, 2], 0))
    wd = both & (o["params"][:, 0] >= 100) & (sg < 5) & (sp < 5)
    dB = np.abs(g["params"][:, 0] - o["params"][:, 0])
    dg = np.abs(g["params"][:, 1] - o["params"][:, 1])
    dp = np.abs((g["params"][:, 2] - o["params"][:, 2] + 90.0) % 180.0 - 90.0)
    out["wd"] = wd
    out["angles_ok"] = (dB <= 1.0) & (dg <= 0.05) & (dp <= 0.05)
    return out


def _equal_counts_agree(c, g, o, obs, w):
    """Pixels converged in both runs with equal iteration counts agree in chi2
    to 1e-3, unless the oracle itself is not reproducible on the pixel: one
    of eight oracle runs on its observations nudged by 1e-7 (relative) ends
    more than 1e-3 from the unnudged chi2.  An equal count is then a
    coincidence of two trajectories that parted (LM on such a pixel lands in
    different minima under perturbations at the FP32 rounding level)."""
    same = c["both"] & (g["iters"] == o["iters"])
    assert same.sum() > 100
    for i in np.flatnonzero(same & (c["rel"] > 1e-3)):
        rng = np.random.default_rng(int(i))
        o1 = np.asarray(obs[i:i + 1], dtype=np.float64)
        spread = 0.0
        for _ in range(8):
            r = lm.invert(o1 * (1.0 + 1e-7 * rng.standard_normal(o1.shape)), w[i:i + 1],
                          f32(T), f32(X), LINE)
            spread = max(spread, abs(r["chi2"][0] / o["chi2"][i] - 1.0))
        assert spread > 1e-3, (int(i), float(c["rel"][i]), spread)


def test_standard_guess_parity(vf):
    """1000 pixels (7 full blocks and a ragged tail) of the small workload."""
    v, h, torch = vf
    p, obs, w = _case(1000, W.SEEDS["small"])
    g = _gpu(v, h, torch, obs, w)
    o = lm.invert(obs, w, f32(T), f32(X), LINE)
    c = _compare(g, o)
    assert c["both"].mean() > 0.5
    assert np.mean(c["rel"][c["both"]] <= 1e-3) >= 0.98
    assert np.mean(c["angles_ok"][c["wd"]]) >= 0.98
    _equal_counts_agree(c, g, o, obs, w)
    assert np.mean(g["status"] == o["status"]) >= 0.8


def test_near_truth_parity_and_covariance(vf):
    v, h, torch = vf
    p, obs, w = _case(512, 1)
    init = p.copy()
    init[:, 0] = init[:, 0] * 1.1 + 20
    init[:, 1] = np.clip(init[:, 1] + 5, 0, 180)
    init = f32(init)
    g = _gpu(v, h, torch, obs, w, init=init)
    o = lm.invert(obs, w, f32(T), f32(X), LINE, init=init)
    c = _compare(g, o)
    assert c["both"].mean() > 0.8
    assert np.mean(c["rel"][c["both"]] <= 1e-3) >= 0.98
    assert np.mean(c["angles_ok"][c["wd"]]) >= 0.98
    # covariance of well-determined pixels: diagonal within 5 % for 98 %
    wd = c["wd"]
    for q in (0, 1, 2, 6):
        r = np.abs(g["cov"][wd, q, q] / o["cov"][wd, q, q] - 1)
        assert np.mean(r <= 0.05) >= 0.98, q


def test_noise_free_recovers_truth(vf):
    v, h, torch = vf
    p, obs, w = _case(256, 2, noise=False)
    init = p.copy()
    init[:, 0] = init[:, 0] * 1.05 + 10
    init[:, 3] *= 1.1
    g = _gpu(v, h, torch, obs, w, init=f32(init), cfg={"max_iter": 100, "conv_rtol": 1e-9})
    strong = (p[:, 0] > 200) & (np.sin(np.radians(p[:, 1])) > 0.3)
    good = g["chi2"] < 1e-2
    assert good.mean() > 0.85
    m = strong & good
    assert np.median(np.abs(g["params"][m, 0] - p[m, 0])) < 0.5
    assert np.median(np.abs(g["params"][m, 1] - p[m, 1])) < 0.02


def test_bad_inputs_and_caps(vf):
    v, h, torch = vf
    p, obs, w = _case(40, 3)
    obs[1, 5] = np.nan
    w[2] = 0.0
    w[3, 0] = np.inf
    init = p.copy()
    init[4, 3] = np.nan
    g = _gpu(v, h, torch, obs, w, init=f32(init))
    assert list(g["status"][1:5]) == [3, 3, 3, 3]
    assert np.all(g["status"][5:] != 3)
    assert np.all(g["cov"][1:5] == 0)
    o = lm.invert(obs, w, f32(T), f32(X), LINE, init=f32(init))
    assert np.array_equal(o["status"][1:5], g["status"][1:5])
    # cap of 0: the model is the (bounded) initial guess, chi2 evaluated there
    g0 = _gpu(v, h, torch, obs[5:], w[5:], cfg={"max_iter": 0})
    o0 = lm.invert(obs[5:], w[5:], f32(T), f32(X), LINE, max_iter=0)
    assert np.all(g0["status"] == 1) and np.all(g0["iters"] == 0)
    np.testing.assert_allclose(g0["params"], o0["params"], rtol=1e-6, atol=1e-5)
    np.testing.assert_allclose(g0["chi2"], o0["chi2"], rtol=1e-4)


def test_held_parameters_and_shared_weights(vf):
    v, h, torch = vf
    p, obs, w = _case(200, 4)
    free = 0x1FF & ~(1 << 5) & ~(1 << 3)   # damping and eta0 held at the initial values
    init = p.copy()
    init[:, 0] += 50
    init = f32(init)
    wshared = w[0].copy()
    g = _gpu(v, h, torch, obs, np.broadcast_to(wshared, w.shape).copy(), init=init,
             cfg={"free_mask": free})
    t = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda:0")  # noqa: E731
    r2 = v.vfisv_invert(h, t(obs), t(wshared), t(T), t(X), LINE, init=t(init),
                        config={"free_mask": free})
    assert np.array_equal(r2["params"].cpu().numpy(), g["params"])
    assert np.array_equal(g["params"][:, 5], init[:, 5])
    assert np.array_equal(g["params"][:, 3], init[:, 3])
    assert np.all(g["cov"][:, 5, :] == 0) and np.all(g["cov"][:, :, 3] == 0)
    o = lm.invert(obs, np.broadcast_to(wshared, w.shape), f32(T), f32(X), LINE, init=init,
                  free_mask=free)
    c = _compare(g, o)
    assert np.mean(c["rel"][c["both"]] <= 1e-3) >= 0.98


def test_host_buffers_match_device(vf):
    v, h, torch = vf
    p, obs, w = _case(300, 5)
    g = _gpu(v, h, torch, obs, w)
    gh = _gpu(v, h, torch, obs, w, host=True)
    for k in ("params", "chi2", "iters", "status", "cov"):
        assert np.array_equal(g[k], gh[k]), k


def test_empty_map(vf):
    v, h, torch = vf
    r = v.vfisv_invert(h, np.zeros((0, 24), np.float32), np.zeros((0, 24), np.float32),
                       T.astype(np.float32), X.astype(np.float32), LINE)
    assert r["params"].shape == (0, 10)


def test_full_map_sampled(vf):
    """The 1024x1024 map inverted in the launch configuration the benchmark
    times; 400 sampled pixels carry oracle-synthesised observations and are
    compared with the oracle's inversion of the same observations."""
    v, h, torch = vf
    npix = 1024 * 1024
    seed = W.SEEDS["map1024"]
    p = f32(W.quiet_and_active_params(npix, seed))
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(a, dtype=torch.float32, device=dev)  # noqa: E731
    syn = v.vfisv_synth(h, t(p), t(T), t(X), LINE).reshape(npix, 24)
    nz = torch.tensor(W.noise(npix, 24, seed), dtype=torch.float32, device=dev)
    sig = 1e-3 * (t(p[:, 7]) + t(p[:, 8]))[:, None]
    obs = syn + sig * nz
    w = (1.0 / (sig * sig)).expand(npix, 24).contiguous()
    idx = np.sort(np.random.default_rng(1).choice(npix, 400, replace=False))
    s_or = me.synth(p[idx], f32(T), f32(X), LINE).reshape(len(idx), 24)
    o_obs, o_w = W.observe(s_or, p[idx], W.noise(npix, 24, seed)[idx])
    o_obs, o_w = f32(o_obs), f32(o_w)
    obs[torch.tensor(idx, device=dev)] = t(o_obs)
    w[torch.tensor(idx, device=dev)] = t(o_w)
    r = v.vfisv_invert(h, obs.contiguous(), w, t(T), t(X), LINE)
    v.vfisv_check(h)
    g = {k: x.cpu().numpy()[idx] for k, x in r.items()}
    o = lm.invert(o_obs, o_w, f32(T), f32(X), LINE)
    c = _compare(g, o)
    assert c["both"].mean() > 0.4
    assert np.mean(c["rel"][c["both"]] <= 1e-3) >= 0.95
    st = r["status"].cpu().numpy()
    assert np.all((st >= 0) & (st <= 2))


def test_work_counters(vf):
    """The LM kernel's work counters (vfisv_counters): one pass per trial plus
    one per starting model, every pixel retired, the packed table's 63 kept
    grid points per pass, and accepted trials close to the oracle's count of
    successful steps on the same inputs (trajectories part at near ties)."""
    v, h, torch = vf
    p, obs, w = _case(2000, 61)
    v.vfisv_counters(h, reset=True)
    g = _gpu(v, h, torch, obs, w)
    c = v.vfisv_counters(h, reset=True)
    assert c["retired"] == 2000
    assert c["passes"] == int(g["iters"].sum()) + 2000
    assert c["points"] == 63 * c["passes"]
    o = lm.invert(obs, w, f32(T), f32(X), LINE)
    assert abs(c["accepted"] / o["accepted"].sum() - 1) < 0.03, (c, o["accepted"].sum())
    assert v.vfisv_counters(h)["passes"] == 0  # reset


@pytest.mark.parametrize("tpp,block", [(2, 64), (2, 256), (4, 128)])
def test_threads_per_pixel_parity(vf, tpp, block):
    """Several threads per pixel (the lanes of a pixel split its wavelength
    points and add their sums by shuffles) meet the same parity criteria
    against the oracle as one thread per pixel, on 1000 pixels of the small
    workload; the work counters still count each pixel once."""
    v, h, torch = vf
    p, obs, w = _case(1000, W.SEEDS["small"])
    v.vfisv_set_launch_shape(h, block, tpp)
    try:
        v.vfisv_counters(h, reset=True)
        g = _gpu(v, h, torch, obs, w)
        c_ = v.vfisv_counters(h, reset=True)
    finally:
        v.vfisv_set_launch_shape(h, 128, 1)
    assert c_["retired"] == 1000 and c_["passes"] == int(g["iters"].sum()) + 1000
    o = lm.invert(obs, w, f32(T), f32(X), LINE)
    c = _compare(g, o)
    assert c["both"].mean() > 0.5
    assert np.mean(c["rel"][c["both"]] <= 1e-3) >= 0.98
    assert np.mean(c["angles_ok"][c["wd"]]) >= 0.98
    _equal_counts_agree(c, g, o, obs, w)
