"""Randomised restarts (Sec. 4.2) on the GPU vs the oracle.

* The perturbation (SplitMix64 draws, amplitudes, bounds) matches the
  oracle's for every model: the same 53-bit uniforms on both sides, so the
  only differences are FP32 roundings (B, eta0, dlambdaD, a, v within 2 ulp
  of the oracle's value rounded to FP32; the angles, whose reflections and
  wrap-arounds run in FP32 near 180-360 deg where one ulp is 1.5-3e-5 deg,
  within 4e-5 deg, psi modulo 180).
* Inversions with restarts: each pixel's trajectory is plain LM until its
  first restart, then a chain of segments whose triggers are decided by
  chi2 comparisons, so GPU and oracle runs part where FP32 and FP64 chi2 tie
  differently.  Compared is what is unique: the iteration count (exactly
  max_iter), chi2 where the chains are well conditioned (started near the
  true model), agreement no worse than the oracle's own under a 1e-7 input
  nudge for the full rule, and the restart result never above plain LM's
  with restarts only at convergence.
* What restarts buy (the paper's motivation, escaping local minima) is
  measured on the GPU with a generous budget of 100 iterations.
"""
import numpy as np
import pytest

import workloads as W
from oracle import lm, me
from gpu_common import LINE, T, X, f32, vf  # noqa: F401

pytestmark = pytest.mark.gpu
FREE = np.array([(0x1FF >> k) & 1 for k in range(10)], dtype=bool)


def _case(n, seed, fastflow=False):
    p = W.quiet_and_active_params(n, seed)
    if fastflow:  # strong fields with large line-of-sight velocities
        g = np.random.default_rng(seed)
        p[:, 6] = g.uniform(2.5, 6.0, n) * np.sign(g.uniform(-1, 1, n))
        p[:, 0] = g.uniform(1500, 3000, n)
    p = f32(p)
    s = me.synth(p, f32(T), f32(X), LINE).reshape(n, -1)
    obs, w = W.observe(s, p, W.noise(n, 24, seed))
    return p, f32(obs), f32(w)


def _gpu(v, h, torch, obs, w, init=None, **cfg):
    t = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda:0")  # noqa: E731
    r = v.vfisv_invert(h, t(obs), t(w), t(T), t(X), LINE,
                       init=None if init is None else t(init), config=cfg)
    v.vfisv_check(h)
    return {k: (x.cpu().numpy() if x is not None else None) for k, x in r.items()}


@pytest.mark.parametrize("k,mask", [(1, 0x1FF), (2, 0x1FF), (7, 0x1FF), (3, 0x1FF & ~0x41)])
def test_restart_models_vs_oracle(vf, k, mask):
    v, h, torch = vf
    n = 4096
    m = f32(W.quiet_and_active_params(n, 60 + k))
    free = np.array([(mask >> j) & 1 for j in range(10)], dtype=bool)
    got = v.vfisv_restart_models(h, m.astype(np.float32), 1000, k, free_mask=mask, seed=12345)
    ref = lm.restart_model(m, 1000 + np.arange(n), k, 12345, free)
    ref32 = ref.astype(np.float32)
    for p in (0, 3, 4, 5, 6, 7, 8, 9):
        ulp = np.spacing(np.abs(ref32[:, p]))
        bad = np.abs(got[:, p] - ref32[:, p]) > 2 * ulp + 1e-30
        assert not bad.any(), (p, np.flatnonzero(bad)[:5], got[bad, p][:5], ref[bad, p][:5])
    assert np.abs(got[:, 1] - ref[:, 1]).max() <= 4e-5
    dpsi = np.abs((got[:, 2] - ref[:, 2] + 90.0) % 180.0 - 90.0)
    assert dpsi.max() <= 4e-5
    # held parameters are copied
    for p in np.flatnonzero(~free):
        assert np.array_equal(got[:, p], m[:, p].astype(np.float32))


def test_restarts_near_truth_parity(vf):
    """Started near the true model, segment 0 converges on both sides at the
    same iteration and every restart starts from the same best model with the
    same draws: chi2 within 1e-3 for >= 95 % of the pixels (the oracle
    against itself with the observations nudged by 1e-7 relative: 98.7 %)."""
    v, h, torch = vf
    p, obs, w = _case(384, 61)
    init = p.copy()
    init[:, 0] *= 1.1
    init[:, 3] *= 1.2
    kw = dict(max_iter=30, restarts=1, seed=77)
    g = _gpu(v, h, torch, obs, w, init=init, **kw)
    o = lm.invert(obs, w, f32(T), f32(X), LINE, init=init, **kw)
    assert np.all(g["iters"] == 30) and np.all(o["iters"] == 30)
    rel = np.abs(g["chi2"] / o["chi2"] - 1)
    print(f"near truth: chi2 within 1e-3 {np.mean(rel <= 1e-3):.3f}, status agree "
          f"{np.mean(g['status'] == o['status']):.3f}, restarted {np.mean(o['restarts'] > 0):.3f}")
    assert np.mean(o["restarts"] > 0) > 0.7
    assert np.mean(rel <= 1e-3) >= 0.95
    # the status is the 1e-4 convergence test in any segment, taken on FP32
    # synthesis on the GPU: borderline tests flip more often than in one run
    assert np.mean(g["status"] == o["status"]) >= 0.9


def test_full_rule_vs_oracle_sensitivity(vf):
    """The paper's full rule from the standard guess: the restart chains are
    sensitive to rounding (a tie broken differently changes every later
    segment), so the GPU must agree with the oracle about as well as the
    oracle agrees with itself under a 1e-7 relative nudge of the
    observations (within 0.08), and its chi2 is Eq. 1 at its own model."""
    v, h, torch = vf
    p, obs, w = _case(384, 61)
    kw = dict(max_iter=30, restarts=7, seed=77)
    g = _gpu(v, h, torch, obs, w, **kw)
    o = lm.invert(obs, w, f32(T), f32(X), LINE, **kw)
    nudged = obs * (1 + 1e-7 * np.random.default_rng(0).standard_normal(obs.shape))
    o2 = lm.invert(nudged, w, f32(T), f32(X), LINE, **kw)
    assert np.all(g["iters"] == 30) and np.all(o["iters"] == 30)
    agree = np.mean(np.abs(g["chi2"] / o["chi2"] - 1) <= 1e-3)
    self_agree = np.mean(np.abs(o2["chi2"] / o["chi2"] - 1) <= 1e-3)
    print(f"full rule: GPU-oracle {agree:.3f}, oracle-nudged oracle {self_agree:.3f}")
    assert agree >= self_agree - 0.08
    assert abs(np.median(g["chi2"]) / np.median(o["chi2"]) - 1) < 0.02
    syn = me.synth(f32(g["params"]), f32(T), f32(X), LINE).reshape(len(p), -1)
    np.testing.assert_allclose(lm.chi2(obs, syn, w, 9), g["chi2"], rtol=2e-4)


def test_restart_at_convergence_never_worse(vf):
    v, h, torch = vf
    p, obs, w = _case(2048, 62)
    a = _gpu(v, h, torch, obs, w, max_iter=40)
    b = _gpu(v, h, torch, obs, w, max_iter=40, restarts=1, seed=5)
    assert np.all(b["chi2"] <= a["chi2"] * (1 + 1e-5))
    assert np.all(b["iters"] == 40)
    conv = a["status"] == 0
    assert np.all(b["status"][conv] == 0)
    # covariance of the best model: finite, positive variances for free parameters
    ok = b["status"] != 3
    d = np.diagonal(b["cov"][ok], axis1=1, axis2=2)[:, :9]
    assert np.all(np.isfinite(d)) and np.mean(d > 0) > 0.99


@pytest.mark.parametrize("fastflow", [False, True])
def test_restarts_bad_fit_fractions(vf, fastflow):
    """With 100 iterations: restarts only at convergence never leave more
    pixels far (1.5x) above the fit started at the true model than plain LM;
    on the uniform mix the paper's rule (7) and (b) with restarts at
    convergence (5) leave fewer (measured: 5.2 % -> 4.0 %).  On strong
    fields with fast flows trigger (b) interrupts slow but progressing
    descents and the full rule leaves more (7.5 % -> 8.3 %): reported, not
    asserted."""
    v, h, torch = vf
    n = 16384
    p, obs, w = _case(n, 63 + fastflow, fastflow)
    ref = _gpu(v, h, torch, obs, w, init=p, max_iter=100, conv_rtol=1e-8)["chi2"]
    plain = _gpu(v, h, torch, obs, w, max_iter=100)["chi2"]
    res = {}
    for mask in (1, 5, 7):
        r = _gpu(v, h, torch, obs, w, max_iter=100, restarts=mask, seed=21)["chi2"]
        res[mask] = np.mean(r > 1.5 * ref)
    bad_plain = np.mean(plain > 1.5 * ref)
    print(f"fastflow={fastflow}: bad fits plain {bad_plain:.4f} restarts " +
          " ".join(f"{m}:{b:.4f}" for m, b in res.items()))
    assert res[1] <= bad_plain
    if not fastflow:
        assert res[5] < bad_plain and res[7] < bad_plain
