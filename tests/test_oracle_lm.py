"""Pins of the FP64 oracle's Levenberg-Marquardt inversion.

Each test ties the oracle to something other than itself: the printed
Table 2, closed-form linear least squares where the model is linear,
noise-free round trips, chi-square statistics of Gaussian noise, a
brute-force grid search, and the sample scatter of repeated noise draws.
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import lm, me

GOLD = os.path.join(os.path.dirname(__file__), "golden")
X = W.wavelength_grid()
T = W.hmi_filters(X)
LINE = W.FE6173


def _obs(n, seed, noise=True):
    p = W.quiet_and_active_params(n, seed)
    s = me.synth(p, T, X, LINE).reshape(n, -1)
    nz = W.noise(n, s.shape[1], seed) if noise else np.zeros_like(s)
    o, w = W.observe(s, p, nz)
    return p, s, o, w


def test_table2_golden():
    rows = np.loadtxt(os.path.join(GOLD, "table2_eps.txt"))
    got = lm.eps_update(rows[:, 0], rows[:, 1] > 0.5)
    np.testing.assert_allclose(got, rows[:, 2], rtol=1e-12)


def test_chi2_definition_eq1():
    # (4L - F) normalisation with L = 6 positions and F = 9 free parameters
    obs = np.ones((1, 24))
    syn = np.zeros((1, 24))
    w = np.full((1, 24), 4.0)
    assert lm.chi2(obs, syn, w, 9)[0] == pytest.approx(24 * 4.0 / 15)


def test_linear_parameters_closed_form():
    """S0 and S1 enter the model linearly: with only they free, one undamped
    Gauss-Newton step lands on the linear least-squares solution."""
    p, s, o, w = _obs(16, 21)
    init = p.copy()
    init[:, 7] *= 0.5
    init[:, 8] *= 1.4
    free = (1 << 7) | (1 << 8)
    r = lm.invert(o, w, T, X, LINE, init=init, max_iter=1, eps0=1e-12, free_mask=free)
    base = p.copy()
    base[:, 7], base[:, 8] = 1.0, 0.0
    c0 = me.synth(base, T, X, LINE).reshape(16, -1)
    base[:, 7], base[:, 8] = 0.0, 1.0
    c1 = me.synth(base, T, X, LINE).reshape(16, -1)
    for i in range(16):
        A = np.stack([c0[i], c1[i]], 1) * np.sqrt(w[i])[:, None]
        sol = np.linalg.lstsq(A, o[i] * np.sqrt(w[i]), rcond=None)[0]
        np.testing.assert_allclose(r["params"][i, 7:9], sol, rtol=1e-9)


def test_noise_free_round_trip():
    p, s, o, w = _obs(24, 22, noise=False)
    init = p.copy()
    init[:, 0] = init[:, 0] * 1.05 + 10
    init[:, 1] = np.clip(init[:, 1] + 3, 0, 180)
    init[:, 3] *= 1.1
    init[:, 6] += 0.2
    r = lm.invert(o, w, T, X, LINE, init=init, max_iter=200, conv_rtol=1e-12)
    assert np.median(r["chi2"]) < 1e-8
    good = r["chi2"] < 1e-8
    assert good.mean() > 0.9
    strong = good & (p[:, 0] > 100) & (np.sin(np.radians(p[:, 1])) > 0.2)
    np.testing.assert_allclose(r["params"][strong, 0], p[strong, 0], rtol=1e-4)
    np.testing.assert_allclose(r["params"][strong, 1], p[strong, 1], atol=1e-3)
    dpsi = np.abs((r["params"][strong, 2] - p[strong, 2] + 90.0) % 180.0 - 90.0)
    assert dpsi.max() < 1e-3


def test_chi2_statistics_with_noise():
    """Gaussian noise of the stated sigma: E[chi2(true)] = 24/15 and at the
    fitted minimum E[chi2] = (24 - 9)/15 = 1 (Eq. 1 normalisation)."""
    p, s, o, w = _obs(256, 23)
    c_true = lm.chi2(o, s, w, 9)
    assert abs(c_true.mean() - 24 / 15) < 0.12
    r = lm.invert(o, w, T, X, LINE, init=p, max_iter=60, conv_rtol=1e-8)
    ok = r["status"] == lm.CONVERGED
    assert ok.mean() > 0.8
    assert np.all(r["chi2"] <= c_true + 1e-12)
    assert abs(r["chi2"][ok].mean() - 1.0) < 0.12


def test_minimum_vs_grid_search():
    """A brute-force scan over (B, gamma, psi) around the LM result finds no
    lower chi2 (other parameters at the LM values)."""
    p, s, o, w = _obs(4, 24)
    p[:, 0] = np.maximum(p[:, 0], 800.0)
    s = me.synth(p, T, X, LINE).reshape(4, -1)
    o, w = W.observe(s, p, W.noise(4, 24, 24))
    r = lm.invert(o, w, T, X, LINE, init=p, max_iter=100, conv_rtol=1e-10)
    for i in range(4):
        m = r["params"][i]
        grid = []
        for dB in np.linspace(-30, 30, 7):
            for dg in np.linspace(-3, 3, 7):
                for dp in np.linspace(-3, 3, 7):
                    q = m.copy()
                    q[0] += dB
                    q[1] += dg
                    q[2] += dp
                    grid.append(q)
        grid = np.array(grid)
        c = lm.chi2(o[i:i + 1].repeat(len(grid), 0), me.synth(grid, T, X, LINE).reshape(len(grid), -1),
                    w[i:i + 1].repeat(len(grid), 0), 9)
        assert r["chi2"][i] <= c.min() + 1e-9


def test_covariance_matches_noise_scatter():
    p = W.quiet_and_active_params(1, 25)
    p[0, 0], p[0, 1], p[0, 3] = 1500.0, 50.0, 8.0
    s = me.synth(p, T, X, LINE).reshape(1, -1)
    n = 300
    P = np.repeat(p, n, 0)
    S = np.repeat(s, n, 0)
    o, w = W.observe(S, P, W.noise(n, 24, 26))
    r = lm.invert(o, w, T, X, LINE, init=P, max_iter=60, conv_rtol=1e-9)
    ok = r["status"] == lm.CONVERGED
    assert ok.mean() > 0.9
    for q in (0, 1, 6):
        sd = r["params"][ok, q].std()
        pred = np.sqrt(r["cov"][ok, q, q].mean())
        assert 0.75 < sd / pred < 1.3, (q, sd, pred)


def test_bad_input_status():
    p, s, o, w = _obs(4, 27)
    o[1, 3] = np.nan
    w[2] = 0.0
    r = lm.invert(o, w, T, X, LINE, max_iter=5)
    assert r["status"][1] == lm.BAD_INPUT and r["status"][2] == lm.BAD_INPUT
    assert r["status"][0] != lm.BAD_INPUT


def test_bounds_equivalences():
    """Negative B with gamma -> 180 - gamma and reflected gamma give the same
    Stokes vector, so the bounds never change the model."""
    p = W.quiet_and_active_params(6, 28)
    q = p.copy()
    q[:, 0] = -q[:, 0]
    q[:, 1] = 180.0 - q[:, 1]
    np.testing.assert_allclose(me.synth(lm.apply_bounds(q), T, X, LINE), me.synth(p, T, X, LINE), atol=1e-13)
    q = p.copy()
    q[:, 1] = -q[:, 1]
    np.testing.assert_allclose(me.synth(q, T, X, LINE), me.synth(lm.apply_bounds(q), T, X, LINE), atol=1e-13)


def test_eq15_limb_darkening_golden():
    rows = np.loadtxt(os.path.join(GOLD, "eq15_icont.txt"))
    for mu, ic in rows:
        assert abs(lm.icont_mu(mu) - ic) < 1e-12
    mu = np.linspace(0.05, 1, 50)
    assert np.all(np.diff(lm.icont_mu(mu)) > 0)   # limb darkening: brighter towards the centre


def test_eq14_weights():
    obs = np.zeros((3, 24))
    obs[:, :6] = np.array([[1.0], [0.5], [0.2]])   # continuum 1, 0.5, 0.2 of disk centre
    w = lm.limb_weights(obs, np.array([1.0, 1.0, 1.0]), 1.0, [1e-3, 1e-3, 1e-3, 1e-3])
    wI = 0.7778 * np.abs(1.0001 - np.array([1.0, 0.5, 0.2])) + 0.3
    np.testing.assert_allclose(w[:, 0], wI ** 2 / 1e-6, rtol=1e-12)
    np.testing.assert_allclose(w[:, 6:], 1e6, rtol=1e-12)
    # quiet Sun (continuum ~ I_cont(mu)) gets w_I ~ 0.3, a dark umbra ~ 1
    assert abs(np.sqrt(w[0, 0] * 1e-6) - 0.3) < 1e-3 and np.sqrt(w[2, 0] * 1e-6) > 0.9


def test_hessian_reuse_off_and_on():
    """hess_reuse = 0 is the plain iteration bit for bit; with reuse the
    iteration still reaches the same minimum (the fixed point of the step
    does not depend on the matrix), and the gradient is exactly the one at
    the final model."""
    p, s, o, w = _obs(48, 29)
    a = lm.invert(o, w, T, X, LINE, max_iter=60)
    b = lm.invert(o, w, T, X, LINE, max_iter=60, hess_reuse=0.0)
    assert np.array_equal(a["params"], b["params"]) and np.array_equal(a["chi2"], b["chi2"])
    c = lm.invert(o, w, T, X, LINE, init=p, max_iter=200, conv_rtol=1e-9)
    d = lm.invert(o, w, T, X, LINE, init=p, max_iter=200, conv_rtol=1e-9, hess_reuse=1e-2)
    both = (c["status"] == lm.CONVERGED) & (d["status"] == lm.CONVERGED)
    assert both.mean() > 0.8
    # with a stale matrix the last steps converge linearly, not quadratically,
    # so the stopping test (1e-9 per step) can end a few steps apart
    np.testing.assert_allclose(d["chi2"][both], c["chi2"][both], rtol=1e-5)


def test_free_filling_factor_round_trip():
    """alpha free (free_mask bit 9): noise-free strong-field profiles with
    alpha in [0.4, 0.9] are recovered from a perturbed start, and freeing
    alpha never ends above the held-alpha fit of data made with alpha = 1."""
    n = 16
    p = W.quiet_and_active_params(n, 30)
    g = np.random.default_rng(30)
    p[:, 0] = g.uniform(1200, 2800, n)
    p[:, 1] = g.uniform(30, 150, n)
    p[:, 9] = g.uniform(0.4, 0.9, n)
    s = me.synth(p, T, X, LINE).reshape(n, -1)
    o, w = W.observe(s, p, np.zeros_like(s))
    init = p.copy()
    init[:, 9] = np.clip(p[:, 9] + 0.15, 0, 1)
    init[:, 0] *= 0.95
    r = lm.invert(o, w, T, X, LINE, init=init, max_iter=200, conv_rtol=1e-12, free_mask=0x3FF)
    good = r["chi2"] < 1e-8
    assert good.mean() > 0.8
    np.testing.assert_allclose(r["params"][good, 9], p[good, 9], atol=1e-4)
    np.testing.assert_allclose(r["params"][good, 0], p[good, 0], rtol=1e-4)
    p1, s1, o1, w1 = _obs(24, 31)
    held = lm.invert(o1, w1, T, X, LINE, init=p1, max_iter=60, conv_rtol=1e-8)
    free = lm.invert(o1, w1, T, X, LINE, init=held["params"], max_iter=60, conv_rtol=1e-8,
                     free_mask=0x3FF)
    assert np.all(free["chi2"] <= held["chi2"] * (1 + 1e-9) * (24 - 9) / (24 - 10) + 1e-12)
    assert np.all((free["params"][:, 9] >= 0) & (free["params"][:, 9] <= 1))


def test_damping_floor_reading_is_not_load_bearing(monkeypatch):
    """The paper gives Table 2 without a floor for eps; the oracle keeps
    eps >= 1e-9.  With a floor of 1e-12 instead, the converged results of the
    standard-guess inversion of the uniform mix barely move: the floor only
    binds after ~20 successes in a row, by which time the convergence test
    has normally stopped the pixel."""
    p, s, o, w = _obs(48, 31)
    r9 = lm.invert(o, w, T, X, LINE, max_iter=50)
    monkeypatch.setattr(lm, "EPS_MIN", 1e-12)
    r12 = lm.invert(o, w, T, X, LINE, max_iter=50)
    both = (r9["status"] == lm.CONVERGED) & (r12["status"] == lm.CONVERGED)
    assert both.mean() > 0.5
    same_st = (r9["status"] == r12["status"]).mean()
    assert same_st >= 0.95
    rel = np.abs(r12["chi2"][both] / r9["chi2"][both] - 1)
    assert (rel < 1e-6).mean() >= 0.95, np.sort(rel)[-5:]
    assert (r9["iters"][both] == r12["iters"][both]).mean() >= 0.95


def _random_blob(seed, obs, params):
    from oracle import mlp
    rng = np.random.default_rng(seed)
    weights = [(rng.uniform(-1, 1, (a, b)) * np.sqrt(6.0 / a), rng.normal(0, 0.05, b))
               for a, b in zip(mlp.LAYERS[:-1], mlp.LAYERS[1:])]
    return mlp.pack(weights, mlp.statistics(obs, params))


def test_mixed_routing_extremes():
    """Confidence routing of the mixed inversion at its two limits: every
    pixel routed gives exactly plain LM from the standard guess; none routed
    gives LM from the network's guess followed by the plain re-inversion of
    the flagged pixels, composed here by hand from lm.invert."""
    from oracle import mlp
    p, s, o, w = _obs(16, 33)
    blob = _random_blob(5, o, p)
    plain = lm.invert(o, w, T, X, LINE, max_iter=30)
    allr = lm.invert_mixed(o, w, T, X, LINE, blob, nn_cap=10, plain_cap=30, conf_route=-np.inf)
    assert allr["routed"].all() and allr["flagged"].all()
    for k in ("params", "chi2", "status", "iters", "accepted", "cov"):
        np.testing.assert_array_equal(allr[k], plain[k])
    none = lm.invert_mixed(o, w, T, X, LINE, blob, nn_cap=10, plain_cap=30, chi2_flag=2.0,
                           flag_unconverged=True, conf_route=np.inf)
    assert not none["routed"].any()
    weights, stats = mlp.unpack(blob)
    y, _ = mlp.forward(weights, mlp.features(o, stats))
    first = lm.invert(o, w, T, X, LINE, init=mlp.decode(y, o, stats), max_iter=10)
    conv = np.isin(first["status"], (lm.CONVERGED, lm.STALLED))
    flag = ~conv | ~(first["chi2"] <= 2.0)
    np.testing.assert_array_equal(none["flagged"], flag.astype(np.int32))
    ids = np.flatnonzero(flag)
    second = lm.invert(o[ids], w[ids], T, X, LINE, max_iter=30)
    exp_chi2 = first["chi2"].copy()
    better = second["chi2"] < first["chi2"][ids]
    exp_chi2[ids[better]] = second["chi2"][better]
    np.testing.assert_array_equal(none["chi2"], exp_chi2)
    np.testing.assert_array_equal(none["iters"][ids], first["iters"][ids] + second["iters"])
    np.testing.assert_array_equal(none["confidence"], y[:, 10])


def test_mixed_routing_splits_by_confidence():
    """A threshold between the confidence outputs routes exactly the pixels
    above it, which end with their plain result."""
    p, s, o, w = _obs(12, 34)
    blob = _random_blob(6, o, p)
    probe = lm.invert_mixed(o, w, T, X, LINE, blob, nn_cap=0, plain_cap=0, conf_route=np.inf)
    k = float(np.median(probe["confidence"]))
    r = lm.invert_mixed(o, w, T, X, LINE, blob, nn_cap=8, plain_cap=20, conf_route=k)
    routed = probe["confidence"] > k
    np.testing.assert_array_equal(r["routed"].astype(bool), routed)
    ids = np.flatnonzero(routed)
    q = lm.invert(o[ids], w[ids], T, X, LINE, max_iter=20)
    ok = np.isfinite(q["chi2"])
    np.testing.assert_array_equal(r["chi2"][ids[ok]], q["chi2"][ok])
    np.testing.assert_array_equal(r["iters"][ids], q["iters"])
