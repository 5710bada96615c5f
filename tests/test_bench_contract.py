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
