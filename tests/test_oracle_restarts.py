"""Pins of the oracle's randomised restarts (Sec. 4.2).

The generator is pinned to its published output sequences, the uniforms to
their distribution, the perturbation to its stated amplitudes, and the
restart logic to what it must leave unchanged: no trigger before the first
restart means the plain Levenberg-Marquardt trajectory, bit for bit, and a
restart only at convergence can never end above plain LM.
"""
import os

import numpy as np

import workloads as W
from oracle import lm, me

GOLD = os.path.join(os.path.dirname(__file__), "golden")
X = W.wavelength_grid()
T = W.hmi_filters(X)
LINE = W.FE6173
FREE = np.array([(0x1FF >> k) & 1 for k in range(10)], dtype=bool)


def _obs(n, seed):
    p = W.quiet_and_active_params(n, seed)
    s = me.synth(p, T, X, LINE).reshape(n, -1)
    o, w = W.observe(s, p, W.noise(n, s.shape[1], seed))
    return p, o, w


def test_splitmix64_published_sequences():
    for line in open(os.path.join(GOLD, "splitmix64.txt")):
        if line.startswith("#") or not line.strip():
            continue
        seed, idx, val = (int(t) for t in line.split())
        assert lm.splitmix64(seed, idx) == val


def test_restart_uniforms_distribution():
    n = 20000
    u = np.array([[lm.restart_uniform(11, pix, 1 + pix % 5, p) for p in range(2)] for pix in range(n)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01
    assert abs(u.var() - 1 / 12) < 0.003
    assert abs(np.corrcoef(u[:, 0], u[:, 1])[0, 1]) < 0.03
    # a different key gives different numbers
    assert lm.restart_uniform(12, 5, 1, 0) != lm.restart_uniform(11, 5, 1, 0)


def test_restart_model_amplitudes():
    m = np.tile([1200.0, 80.0, 90.0, 8.0, 30.0, 0.6, 0.5, 0.3, 0.7, 1.0], (400, 1))
    for k in (1, 2, 3):
        q = lm.restart_model(m, np.arange(400), k, 5, FREE)
        d = q - m
        for p, a in zip((0, 1, 2, 4, 5, 6), (150.0, 10.0, 15.0, 4.0, 0.05, 0.25)):
            assert np.all(np.abs(d[:, p]) <= a * k + 1e-9)
            assert np.abs(d[:, p]).max() > 0.8 * a * k          # spans its range
        assert np.all(np.abs(np.log(q[:, 3] / m[:, 3])) <= 0.25 * k + 1e-12)
        assert np.array_equal(q[:, 7:], m[:, 7:])               # S0, S1, alpha untouched
    held = FREE.copy()
    held[[0, 6]] = False
    q = lm.restart_model(m, np.arange(400), 2, 5, held)
    assert np.array_equal(q[:, [0, 6]], m[:, [0, 6]])
    # the bounds are applied: B near zero turns negative and flips gamma
    m2 = m.copy()
    m2[:, 0] = 10.0
    q = lm.restart_model(m2, np.arange(400), 1, 5, FREE)
    assert q[:, 0].min() >= 0.0 and np.all((q[:, 1] >= 0) & (q[:, 1] <= 180))


def test_no_trigger_means_plain_trajectory():
    """Before any restart fires the run is plain LM step for step."""
    p, o, w = _obs(24, 51)
    kw = dict(max_iter=5, conv_rtol=0.0)  # no convergence, no (a) before iteration 10
    a = lm.invert(o, w, T, X, LINE, **kw)
    b = lm.invert(o, w, T, X, LINE, restarts=7, seed=3, **kw)
    assert np.array_equal(a["params"], b["params"]) and np.array_equal(a["chi2"], b["chi2"])
    assert np.all(b["iters"] == 5) and np.all(b["restarts"] == 0)


def test_restart_at_convergence_never_worse():
    p, o, w = _obs(32, 52)
    a = lm.invert(o, w, T, X, LINE, max_iter=40)
    b = lm.invert(o, w, T, X, LINE, max_iter=40, restarts=1, seed=9)
    assert np.all(b["chi2"] <= a["chi2"])
    assert np.all(b["iters"] == 40)
    # pixels that converged before the last iteration restart, and stay converged
    conv = a["status"] == lm.CONVERGED
    early = conv & (a["iters"] < 40)
    assert early.sum() > 10 and np.all(b["restarts"][early] >= 1)
    assert np.all(b["status"][conv] == lm.CONVERGED)


def test_restart_result_is_consistent():
    """Output chi2 is Eq. 1 at the output model, and never above the initial chi2."""
    p, o, w = _obs(32, 53)
    r = lm.invert(o, w, T, X, LINE, max_iter=30, restarts=7, seed=4)
    syn = me.synth(r["params"], T, X, LINE).reshape(32, -1)
    np.testing.assert_allclose(lm.chi2(o, syn, w, 9), r["chi2"], rtol=1e-10)
    guess = lm.standard_guess(o, 6)
    c0 = lm.chi2(o, me.synth(lm.apply_bounds(guess), T, X, LINE).reshape(32, -1), w, 9)
    assert np.all(r["chi2"] <= c0)
    assert np.all(r["iters"] == 30) and np.mean(r["restarts"] >= 1) > 0.5
    assert set(np.unique(r["status"])) <= {lm.CONVERGED, lm.MAXITER, lm.STALLED}
