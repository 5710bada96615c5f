"""Benchmark: converged pixels/s of the GB300 Milne-Eddington inversion.

Default workload (N=1): the 1024x1024 plain-LM map -- 1,048,576 pixels,
Fe I 6173.34 A (g_eff = 2.5), 149 wavelengths at 10 mA over +-740 mA, 6 HMI-like
filters (24 observables), per-pixel parameters drawn from the uniform
distributions, Gaussian noise sigma = 1e-3 Ic, LM from the standard guess with
a 50-iteration cap, covariance requested.  A step is one vfisv_invert call
over the whole map (synthetic observations already resident in HBM).

With --impl reference the FP64 CPU oracle is timed instead on a bounded
sample of the same workload (that is the only other place it runs here).

Multi-GPU: pixels are independent, so N ranks invert N independent maps
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

NLAM, NF = 149, 6
METRIC = "converged pixels/s on 1 GB300 at oracle-matched chi2: NN-init mixed vs plain LM"
MAXITER = 50

# Algorithmic FP32 flops of one fused pass (synthesis + 6-column Jacobian +
# filtering) per wavelength point, from the op count of the formulas
# (FMA = 2 flops): Faddeeva (Weideman, N=16) 3 x 135, absorption matrix 26,
# Unno-Rachkovsky 31, Stokes filtering 48, Eqs. 8-9 27, Delta partials 13,
# 20 Stokes partials 90, 6 parameter chains 654.
FLOP_PER_LAMBDA = 3 * 135 + 26 + 31 + 48 + 27 + 13 + 90 + 654
# per pass, outside the wavelength loop: model 60, chi2 (FP64) 72, and on an
# accepted pass the compensated normal equations 24 x 54 x 8.
FLOP_PER_PASS = 60
FLOP_PER_ACCEPT = 24 * 54 * 8


def fp32_peak_tflops(sm_mhz: float, nsm: int = 152) -> float:
    """FP32 pipe peak: SMs x 128 FP32 lanes x 2 flops (FMA) x clock."""
    return nsm * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [r for r in self.rows if len(r) >= 9]
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def make_map(npix: int, seed: int):
    p = W.quiet_and_active_params(npix, seed)
    x = W.wavelength_grid(NLAM)
    T = W.hmi_filters(x)
    return p, x, T


def run_ours(args, rank, world):
    import torch

    import paper_0901_2702_gb300 as v
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    side = args.side
    npix = side * side
    seed = W.SEEDS["map1024"] + 1000 * rank
    p, x, T = make_map(npix, seed)
    line = W.FE6173
    h = v.vfisv_create(dev.index)
    tf = torch.tensor(T, dtype=torch.float32, device=dev)
    tx = torch.tensor(x, dtype=torch.float32, device=dev)
    tp = torch.tensor(p, dtype=torch.float32, device=dev)
    syn = v.vfisv_synth(h, tp, tf, tx, line).reshape(npix, 4 * NF)
    nz = torch.tensor(W.noise(npix, 4 * NF, seed), dtype=torch.float32, device=dev)
    sig = (1e-3 * torch.tensor(W.continuum(p), dtype=torch.float32, device=dev))[:, None]
    obs = (syn + sig * nz).contiguous()
    wts = (1.0 / (sig * sig)).expand(npix, 4 * NF).contiguous()
    del syn, nz, tp
    cfg = v.vfisv_config_default(max_iter=MAXITER)
    out = {"params": torch.empty(npix, 10, device=dev), "chi2": torch.empty(npix, device=dev),
           "iters": torch.empty(npix, dtype=torch.int32, device=dev),
           "status": torch.empty(npix, dtype=torch.int32, device=dev),
           "cov": torch.empty(npix, 10, 10, device=dev)}
    stream = torch.cuda.current_stream(dev)

    def step():
        v.vfisv_invert(h, obs, wts, tf, tx, line, config=cfg, out=out, stream=stream)

    for _ in range(args.warmup):
        step()
    v.vfisv_check(h, stream)
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(dev.index)
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    conv = 0
    passes = 0
    accepts_est = 0
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    v.vfisv_check(h, stream)
    ms = e0.elapsed_time(e1) / args.steps
    st = out["status"]
    conv = int(((st == 0) | (st == 2)).sum().item())
    it = out["iters"].to(torch.int64)
    passes = int((it + 1).sum().item())
    if dist:
        import torch.distributed as tdist
        t = torch.tensor([ms], device=dev)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        ms = float(t.item())
        c = torch.tensor([conv], device=dev, dtype=torch.int64)
        tdist.all_reduce(c)
        conv_total = int(c.item())
    else:
        conv_total = conv
    value = conv_total / (ms / 1e3)

    # end to end: the same call with pinned host buffers, copies inside the timed region
    obs_h = obs.cpu().pin_memory()
    wts_h = wts.cpu().pin_memory()
    T32 = tf.cpu().pin_memory()
    x32 = tx.cpu().pin_memory()
    outh = {k: torch.empty(tuple(t_.shape), dtype=t_.dtype).pin_memory() for k, t_ in out.items()}
    v.vfisv_invert(h, obs_h, wts_h, T32, x32, line, config=cfg, out=outh)  # warm staging
    t0 = time.perf_counter()
    ne2e = max(1, min(args.steps, 3))
    for _ in range(ne2e):
        v.vfisv_invert(h, obs_h, wts_h, T32, x32, line, config=cfg, out=outh)
    e2e_s = (time.perf_counter() - t0) / ne2e
    st_h = outh["status"]
    conv_h = int(((st_h == 0) | (st_h == 2)).sum().item())
    h2d = sum(t_.numel() * t_.element_size() for t_ in (obs_h, wts_h, T32, x32))
    d2h = sum(t_.numel() * t_.element_size() for t_ in outh.values())

    flops = passes * (NLAM * FLOP_PER_LAMBDA + FLOP_PER_PASS)
    achieved = flops / (ms / 1e3) / 1e12
    peak = fp32_peak_tflops(2070.0)
    res = {
        "metric": METRIC, "value": value, "unit": "pixels/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded ME parameters, GPU-synthesised Stokes + Gaussian noise)",
        "config": {"workload": f"plain LM, {side}x{side} map, Fe I 6173 A, 6 filters x 149 lambda, "
                               f"cap {MAXITER}, standard initial guess, covariance on",
                   "pixels_per_gpu": npix, "l2": "inputs 192 MB > 129 MB L2 (no flush)",
                   "parallelism": f"replicas x{world}"},
        "converged_fraction": conv / npix, "mean_iterations": float(it.float().mean().item()),
        "e2e": {"value": conv_h / e2e_s * world, "unit": "pixels/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": 2 * args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "note": "FP32 pipe peak = 152 SM x 128 lanes x 2 x 2070 MHz; algorithmic "
                             "flops = passes x (149 x %d + %d)" % (FLOP_PER_LAMBDA, FLOP_PER_PASS)},
        "clocks": clocks,
    }
    h.close()
    return res


def cpu_baseline(args, sample: int):
    """The FP64 oracle timed on the host, on a bounded sample of the same map."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = f"""
import sys, time, json
sys.path.insert(0, {ROOT!r})
import numpy as np, workloads as W
from oracle import me, lm
side = {args.side}; npix = side*side; n = {sample}
p = W.quiet_and_active_params(npix, W.SEEDS['map1024'])
idx = np.linspace(0, npix - 1, n).astype(np.int64)
x = W.wavelength_grid({NLAM}); T = W.hmi_filters(x)
nz = W.noise(npix, 24, W.SEEDS['map1024'])[idx]
s = me.synth(p[idx], T, x, W.FE6173).reshape(n, -1)
obs, w = W.observe(s, p[idx], nz)
t0 = time.perf_counter()
r = lm.invert(obs, w, T, x, W.FE6173, max_iter={MAXITER})
dt = time.perf_counter() - t0
conv = int(np.sum((r['status'] == 0) | (r['status'] == 2)))
print(json.dumps({{'value': conv / dt, 'seconds': dt, 'n': n}}))
"""
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if out.returncode != 0:
        return {"value": None, "unit": "pixels/s", "cores": 1, "kind": "oracle",
                "sample": f"failed: {out.stderr[-300:]}"}
    d = json.loads(out.stdout.strip().splitlines()[-1])
    return {"value": d["value"], "unit": "pixels/s", "cores": 1, "kind": "oracle",
            "sample": f"{d['n']} pixels evenly spaced over the {args.side}x{args.side} map, "
                      f"{d['seconds']:.1f} s, numpy/scipy FP64, 1 thread"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=1024)
    ap.add_argument("--cpu-sample", type=int, default=384)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus if args.gpus == 1 else 1))

    if args.impl == "reference":
        if rank != 0:
            return
        cb = cpu_baseline(args, args.cpu_sample)
        res = {"metric": METRIC, "value": cb["value"], "unit": "pixels/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
               "impl": "reference", "dtype": "f64", "data": "synthetic",
               "config": {"workload": f"plain LM, {args.side}x{args.side} map (bounded sample)"},
               "cpu_baseline": cb,
               "e2e": {"value": cb["value"], "unit": "pixels/s", "h2d_bytes_per_step": 0,
                       "d2h_bytes_per_step": 0}}
        print(json.dumps(res))
        return

    if world > 1:
        import torch
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    res = run_ours(args, rank, world)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            res["cpu_baseline"] = cpu_baseline(args, args.cpu_sample)
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
