"""Initial models from the filtergrams (Sec. 5) on the GPU vs the oracle,
and what they change in the inversion.

Tolerances: the kernel runs in FP32 on the same float32 observables; its
least-squares sums are of a handful of terms, so B is within 1e-3 relative
(+0.5 G), gamma within 0.05 deg and v within 1e-3 km/s (+1e-4 relative);
the azimuth is compared where the wing polarisation is above 1e-5 I_c
(below that atan2 of two rounding-level sums is arbitrary).
"""
import numpy as np
import pytest

import workloads as W
from oracle import init, lm, me, mlp
from gpu_common import LINE, T, X, f32, vf  # noqa: F401

pytestmark = pytest.mark.gpu


def _case(n, seed, noise=True):
    p = f32(W.quiet_and_active_params(n, seed))
    s = me.synth(p, f32(T), f32(X), LINE).reshape(n, -1)
    nz = W.noise(n, 24, seed) if noise else np.zeros((n, 24))
    obs, w = W.observe(s, p, nz)
    return p, f32(obs), f32(w)


@pytest.mark.parametrize("noise", [False, True])
def test_init_models_vs_oracle(vf, noise):
    v, h, torch = vf
    p, obs, w = _case(3000, 80, noise)
    obs[7, 3] = np.nan                                      # one bad pixel
    g = v.vfisv_init_models(h, obs.astype(np.float32), T.astype(np.float32),
                            X.astype(np.float32), LINE)
    good = np.ones(len(p), bool)
    good[7] = False
    assert np.all(np.isnan(g["init"][7])) and np.isnan(g["pol"][7])
    ref = init.initial_models(obs[good], f32(T), f32(X), LINE)
    wf = init.weak_field(obs[good], f32(T), f32(X), LINE)
    gi, gp = g["init"][good].astype(np.float64), g["pol"][good].astype(np.float64)
    np.testing.assert_allclose(gi[:, 0], ref[:, 0], rtol=1e-3, atol=0.5)
    assert np.abs(gi[:, 1] - ref[:, 1]).max() < 0.05
    np.testing.assert_allclose(gi[:, 6], ref[:, 6], rtol=1e-4, atol=1e-3)
    np.testing.assert_allclose(gi[:, [3, 4, 5, 7, 8, 9]], ref[:, [3, 4, 5, 7, 8, 9]], rtol=1e-6)
    np.testing.assert_allclose(gp, wf["pol"], rtol=1e-5)
    c = init.filter_centres(f32(T), f32(X))
    wk = (c - c.mean()) ** 4
    q, u = obs[good, 6:12], obs[good, 12:18]
    strong = np.hypot((q * wk).sum(1), (u * wk).sum(1)) / wk.sum() > 1e-5
    dpsi = np.abs((gi[:, 2] - ref[:, 2] + 90.0) % 180.0 - 90.0)
    assert strong.mean() > 0.5 and dpsi[strong].max() < 0.05


def test_paper_initialisation_in_mixed_pipeline_vs_oracle(vf):
    """vfisv_invert_nn with the paper's combination (wfa_pol = 0.06) vs the
    oracle's mixed inversion with the same network (trained by the oracle)."""
    v, h, torch = vf
    tp, tobs, tw = _case(16384, 46)
    blob = f32(mlp.train(tobs, tp, steps=150, batch=1024, lr0=2e-3, seed=3))
    p, obs, w = _case(600, 81)
    ref = lm.invert_mixed(obs, w, f32(T), f32(X), LINE, blob, nn_cap=20, plain_cap=50,
                          chi2_flag=3.0, flag_unconverged=True, wfa_pol=0.06)
    g = v.vfisv_invert_nn(h, blob.astype(np.float32), obs.astype(np.float32),
                          w.astype(np.float32), T.astype(np.float32), X.astype(np.float32),
                          LINE, config_nn={"max_iter": 20, "wfa_pol": 0.06}, chi2_flag=3.0,
                          flag_unconverged=True)
    assert np.mean(g["flagged"] == ref["flagged"]) >= 0.85
    both = np.isin(g["status"], (0, 2)) & np.isin(ref["status"], (0, 2))
    rel = np.abs(g["chi2"][both] / ref["chi2"][both] - 1)
    assert both.mean() > 0.5 and np.mean(rel <= 1e-3) >= 0.95


def test_initialisation_effects(vf):
    """Plain LM from the weak-field models vs from the standard guess, and
    the network pipeline with and without the paper's combination, on
    65,536 pixels of the uniform mix: reported, with two guards (the
    weak-field start converges at least as often as the standard guess; the
    paper's combination does not lower the converged fraction by more than
    two points)."""
    v, h, torch = vf
    dev = torch.device("cuda:0")
    n = 1 << 16
    t32 = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device=dev)  # noqa: E731
    tf, tx = t32(T), t32(X)
    tp = t32(W.training_params(1 << 20, W.SEEDS["nn_train"]))
    tobs = v.vfisv_synth(h, tp, tf, tx, LINE).reshape(1 << 20, 24)
    gen = torch.Generator(device=dev)
    gen.manual_seed(3)
    tobs = tobs + 1e-3 * (tp[:, 7] + tp[:, 8])[:, None] * torch.randn(1 << 20, 24, device=dev,
                                                                      generator=gen)
    blob = v.vfisv_nn_init(h, tobs, tp, seed=11)
    v.vfisv_nn_train(h, blob, tobs, tp, batch=8192, epochs=4, lr0=1e-3, seed=12)
    p = t32(W.quiet_and_active_params(n, 82))
    s = v.vfisv_synth(h, p, tf, tx, LINE).reshape(n, 24)
    sig = 1e-3 * (p[:, 7] + p[:, 8])[:, None]
    obs = (s + sig * t32(W.noise(n, 24, 82))).contiguous()
    wts = (1.0 / (sig * sig)).expand(n, 24).contiguous()
    conv = lambda r: torch.isin(r["status"], torch.tensor([0, 2], device=dev)).float().mean().item()  # noqa: E731
    std = v.vfisv_invert(h, obs, wts, tf, tx, LINE)
    wfa = v.vfisv_invert(h, obs, wts, tf, tx, LINE,
                         init=v.vfisv_init_models(h, obs, tf, tx, LINE)["init"])
    nn0 = v.vfisv_invert_nn(h, blob, obs, wts, tf, tx, LINE, chi2_flag=3.0)
    nn1 = v.vfisv_invert_nn(h, blob, obs, wts, tf, tx, LINE, config_nn={"max_iter": 20, "wfa_pol": 0.06},
                            chi2_flag=3.0)
    v.vfisv_check(h)
    it = lambda r: r["iters"].float().mean().item()  # noqa: E731
    print(f"plain std guess: conv {conv(std):.4f} iters {it(std):.2f} | weak-field init: conv "
          f"{conv(wfa):.4f} iters {it(wfa):.2f} | NN: conv {conv(nn0):.4f} iters {it(nn0):.2f} | "
          f"NN + paper combination: conv {conv(nn1):.4f} iters {it(nn1):.2f}")
    assert conv(wfa) >= conv(std) - 0.005
    assert conv(nn1) >= conv(nn0) - 0.02


def test_weak_field_start_parity(vf):
    """vfisv_invert started from the filtergram models (wfa_pol > 0, no
    init) vs the oracle started from its own filtergram models: the same
    criteria as the standard-guess parity test."""
    v, h, torch = vf
    p, obs, w = _case(1000, 83)
    t = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device="cuda:0")  # noqa: E731
    r = v.vfisv_invert(h, t(obs), t(w), t(T), t(X), LINE, config={"wfa_pol": 1.0})
    v.vfisv_check(h)
    g = {k: x.cpu().numpy() for k, x in r.items()}
    o = lm.invert(obs, w, f32(T), f32(X), LINE, wfa_pol=1.0)
    both = np.isin(g["status"], (0, 2)) & np.isin(o["status"], (0, 2))
    rel = np.abs(g["chi2"][both] / o["chi2"][both] - 1)
    print(f"weak-field start: converged in both {both.mean():.3f}, chi2 within 1e-3 {np.mean(rel <= 1e-3):.3f}")
    assert both.mean() > 0.6 and np.mean(rel <= 1e-3) >= 0.98
