"""The benchmark's reference arm (the FP64 oracle on the host cores) keeps the
JSON contract of the GPU arm: one line on rank 0 with the same metric, unit,
direction and workload config, plus the oracle's cpu_baseline and an e2e
object without host-device traffic; the other ranks print nothing."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _run(extra_env=None):
    env = dict(os.environ, **(extra_env or {}))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--steps", "1", "--warmup", "0", "--cpu-sample", "8"],
                          capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)


def test_reference_line():
    import bench

    r = _run()
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "pixels/s" and d["higher_is_better"] is True and d["value"] > 0
    ours = bench.workload_config("disk", 13457608, 1)
    assert d["config"]["workload"] == ours["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert "8 pixels" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "pixels/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_other_ranks_silent():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_calibration_emulates_the_mixed_inversion():
    """The benchmark chooses the routing threshold from two deterministic
    ingredients (LM from the network's guess, plain LM) without rerunning the
    mixed pipeline; its composition must give the oracle's mixed inversion
    for every threshold: the routed pixels' plain result, the others' first
    result unless flagged, then the lower chi2."""
    import numpy as np
    import torch

    import bench
    import workloads as W
    from oracle import lm, me, mlp

    x = W.wavelength_grid()
    T = W.hmi_filters(x)
    p = W.quiet_and_active_params(12, 71)
    s = me.synth(p, T, x, W.FE6173).reshape(12, -1)
    o, w = W.observe(s, p, W.noise(12, 24, 71))
    rng = np.random.default_rng(2)
    weights = [(rng.uniform(-1, 1, (a, b)) * np.sqrt(6.0 / a), rng.normal(0, 0.05, b))
               for a, b in zip(mlp.LAYERS[:-1], mlp.LAYERS[1:])]
    blob = mlp.pack(weights, mlp.statistics(o, p))
    wq, st = mlp.unpack(blob)
    y, _ = mlp.forward(wq, mlp.features(o, st))
    first = lm.invert(o, w, T, x, W.FE6173, init=mlp.decode(y, o, st), max_iter=8)
    plain = lm.invert(o, w, T, x, W.FE6173, max_iter=15)
    tt = lambda r: {"chi2": torch.tensor(r["chi2"]), "status": torch.tensor(r["status"])}  # noqa: E731
    conf = torch.tensor(y[:, 10])
    for k in (-np.inf, float(np.median(y[:, 10])), np.inf):
        ref = lm.invert_mixed(o, w, T, x, W.FE6173, blob, nn_cap=8, plain_cap=15, chi2_flag=1.5,
                              flag_unconverged=True, conf_route=k)
        c2, st_, ran = bench.mixed_outcome(conf > k, tt(first), tt(plain), 1.5, True)
        ok = np.isfinite(ref["chi2"])
        np.testing.assert_array_equal(c2.numpy()[ok], ref["chi2"][ok])
        np.testing.assert_array_equal(st_.numpy()[ok], ref["status"][ok])
        np.testing.assert_array_equal(ran.numpy(), ref["flagged"].astype(bool))
