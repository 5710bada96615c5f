"""Parity on the workload the benchmark times: the 4096x4096 full-disk map
(90 % quiet Sun with B ~ U[0,200] G, active-region blobs up to 3500 G).

A sample of pixels evenly spaced over the disk (quiet Sun and active
regions in their map proportions) is synthesised by the oracle, noised and
rounded to float32, then inverted by the GPU and by the FP64 oracle:
  * plain LM from the standard guess, cap 50 (the plain leg of the bench);
  * the mixed pipeline with the bench's settings for the disk (network
    guess, LM cap 50, plain re-inversion of pixels that did not converge or
    end with chi2 > 2.5, confidence routing) against the oracle's mixed
    inversion with the same network -- trained by the oracle itself, so no
    oracle input comes from the CUDA path -- and the network evaluated with
    the kernel's bfloat16 operand rounding, so that routing and flagging are
    decided in the same precision on both sides.
Each test prints the per-parameter error table (max / p99 / median |delta|
for the nine free parameters and chi2, fraction within the stated
tolerances).  LM is an iteration, and the quiet Sun is ill-conditioned (a
weak field leaves B, gamma, psi nearly free, and six filter samples leave
eta0, dlambdaD, S0, S1 a shallow valley): FP32 synthesis against FP64 parts
trajectories at near ties, after which the two runs take different numbers
of steps and stop at different points.  Measured on this sample, the FP64
oracle against itself with the observations nudged by 1e-7 or 1e-6
relative (Gaussian) agrees on chi2 within 1e-3 for 97.0-97.5 % of the
pixels converged in both, on the status for 91.4-92.7 %, on the field of
the well-determined pixels for 99.3-100 %; the GPU against the oracle
measures 94.6 %, 89.3 % and 98.3 % (FP32 perturbs every iteration, a nudge
only the input).  The bars below sit under those measurements, and every
chi2 mismatch between pixels converged in both must be a trajectory split
(a different iteration count) or a near tie (chi2 within 1e-2).
"""
import numpy as np
import pytest

import oracle_pool
import parity
import workloads as W
from gpu_common import LINE, T, X, f32, vf  # noqa: F401
from oracle import lm, me, mlp

pytestmark = pytest.mark.gpu

N = 1536
PLAIN_CAP, NN_CAP, CHI2_FLAG = 50, 50, 2.5


@pytest.fixture(scope="module")
def disk_sample():
    p, _ = W.full_disk_params(W.SEEDS["disk"])
    idx = np.linspace(0, p.shape[0] - 1, N).astype(np.int64)
    p = f32(p[idx])
    s = me.synth(p, f32(T), f32(X), LINE).reshape(N, -1)
    obs, w = W.observe(s, p, W.noise(N, 24, 900))
    return p, f32(obs), f32(w)


@pytest.fixture(scope="module")
def oracle_plain(disk_sample):
    p, obs, w = disk_sample
    return oracle_pool.run("invert", obs, w, f32(T), f32(X), LINE, max_iter=PLAIN_CAP)


def test_plain_lm_full_disk_vs_oracle(vf, disk_sample, oracle_plain):
    v, h, torch = vf
    p, obs, w = disk_sample
    ref = oracle_plain
    g = v.vfisv_invert(h, obs.astype(np.float32), w.astype(np.float32), T.astype(np.float32),
                       X.astype(np.float32), LINE, config={"max_iter": PLAIN_CAP})
    v.vfisv_check(h)
    tab = parity.error_table(g, ref, parity.well_determined(ref))
    print("\nplain LM, full-disk sample:\n" + parity.format_table(tab))
    assert tab["converged_both"] >= 0.35 * N
    assert np.mean(g["status"] == ref["status"]) >= 0.87
    _splits_or_near_ties(g, ref)
    assert tab["chi2_within_tol"] >= 0.93
    assert tab["field_within_tol_well_determined"] >= 0.97


def test_mixed_pipeline_full_disk_vs_oracle(vf, disk_sample, oracle_plain):
    v, h, torch = vf
    p, obs, w = disk_sample
    tp, tobs, _ = _training_set(16384, 46)
    blob = f32(mlp.train(tobs, tp, steps=150, batch=1024, lr0=2e-3, seed=3))
    weights, st = mlp.unpack(blob)
    y, _ = mlp.forward(weights, mlp.features(obs, st), operand_round=mlp.round_bf16)
    conf_ref = y[:, mlp.NOUT_PARAM]
    k = float(np.median(conf_ref))  # half the pixels routed: both branches run
    ref = oracle_pool.run("invert_mixed", obs, w, f32(T), f32(X), LINE, blob, nn_cap=NN_CAP,
                          plain_cap=PLAIN_CAP, chi2_flag=CHI2_FLAG, flag_unconverged=True,
                          conf_route=k, operand_round=mlp.round_bf16)
    b32, o32 = blob.astype(np.float32), obs.astype(np.float32)
    conf = v.vfisv_nn_infer(h, b32, o32, LINE)["conf"].astype(np.float64)
    g = v.vfisv_invert_nn(h, b32, o32, w.astype(np.float32), T.astype(np.float32),
                          X.astype(np.float32), LINE, config_nn={"max_iter": NN_CAP},
                          config_plain={"max_iter": PLAIN_CAP}, chi2_flag=CHI2_FLAG,
                          flag_unconverged=True, conf_route=k)
    v.vfisv_check(h)
    # the confidence output in the kernel's precision, and the routing it decides
    assert np.median(np.abs(conf - conf_ref)) < 1e-3
    clear = np.abs(conf_ref - k) > 0.02
    assert np.array_equal((conf > k)[clear], (conf_ref > k)[clear])
    assert np.all(g["flagged"][(conf > k)] == 1)
    assert np.mean(g["flagged"] == ref["flagged"]) >= 0.9
    tab = parity.error_table(g, ref, parity.well_determined(ref))
    print("\nmixed pipeline (bench disk settings), full-disk sample:\n" + parity.format_table(tab))
    assert tab["converged_both"] >= 0.35 * N
    _splits_or_near_ties(g, ref)
    assert tab["chi2_within_tol"] >= 0.93
    # routed pixels carry the GPU's plain result bit for bit; against the
    # oracle's plain LM the mixed result meets the headline's chi2 criterion
    # at least as often as the GPU's own plain run does
    gp = v.vfisv_invert(h, o32, w.astype(np.float32), T.astype(np.float32),
                        X.astype(np.float32), LINE, config={"max_iter": PLAIN_CAP})
    routed = conf > k
    for key in ("params", "chi2", "status"):
        assert np.array_equal(g[key][routed], gp[key][routed]), key
    le = np.asarray(g["chi2"], dtype=np.float64) <= oracle_plain["chi2"] * (1 + 1e-3)
    le_p = np.asarray(gp["chi2"], dtype=np.float64) <= oracle_plain["chi2"] * (1 + 1e-3)
    print(f"chi2 <= oracle plain chi2 (1 + 1e-3): mixed {le.mean():.4f}, GPU plain "
          f"{le_p.mean():.4f}; routed {routed.mean():.3f}, flagged {np.mean(g['flagged']):.3f}")
    assert le.mean() >= le_p.mean() - 0.01


def _training_set(n, seed):
    p = f32(W.training_params(n, seed))
    s = me.synth(p, f32(T), f32(X), LINE).reshape(n, -1)
    obs, w = W.observe(s, p, W.noise(n, 24, seed))
    return p, f32(obs), f32(w)


def _splits_or_near_ties(g, ref):
    """Every chi2 mismatch (> 1e-3 relative) between pixels CONVERGED in both
    runs is a trajectory split (different iteration counts) or a near tie
    (within 1e-2)."""
    both = (g["status"] == 0) & (ref["status"] == 0)
    rel = np.abs(np.asarray(g["chi2"], dtype=np.float64) / ref["chi2"] - 1)
    same = g["iters"] == ref["iters"]
    assert np.all(rel[both & same] <= 1e-2), np.sort(rel[both & same])[-3:]
