"""One inference of the initial-guess network over a seeded synthetic map on
the GPU: the small, self-contained launch that profiles of the fused
tensor-core inference kernel capture.

Profiles are synthesised by the library (uniform parameter distributions of
the training set, Fe I 6173 A, 6 filters x 149 wavelengths, noise 1e-3 Ic);
the network has the library's random initial weights and the statistics of
the map.  Prints one JSON line with the time of the timed inference (CUDA
events, after --warmup untimed ones) and its throughput in FLOP/s counted
over the unpadded layers (2 x (24x256 + 2x256x256 + 256x11) per pixel).

    python -m paper_0901_2702_gb300.nn_bench --npix 4194304

With --train it times vfisv_nn_train instead: --epochs passes over the
--npix profiles in batches of --batch, reported per Adam step and as FLOP/s
over the unpadded products of a step (forward, input gradients of layers
1-3, weight gradients: 827,904 flops per sample).

    python -m paper_0901_2702_gb300.nn_bench --train --npix 1048576 --epochs 2
"""
from __future__ import annotations

import argparse
import json
import os
import sys

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

FLOP_PER_PIXEL = 2 * (24 * 256 + 2 * 256 * 256 + 256 * 11)
# one training sample: forward, input gradients of layers 3..1, weight gradients
FLOP_PER_TRAIN_SAMPLE = FLOP_PER_PIXEL + 2 * (256 * 11 + 2 * 256 * 256) + FLOP_PER_PIXEL


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--npix", type=int, default=1 << 22)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--iters", type=int, default=10)
    ap.add_argument("--train", action="store_true", help="time training instead of inference")
    ap.add_argument("--epochs", type=int, default=2)
    ap.add_argument("--batch", type=int, default=8192)
    args = ap.parse_args()

    import numpy as np
    import torch

    import paper_0901_2702_gb300 as v
    import workloads as W

    dev = torch.device("cuda:0")
    h = v.vfisv_create(0)
    t32 = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device=dev)  # noqa: E731
    x = W.wavelength_grid()
    tf, tx = t32(W.hmi_filters(x)), t32(x)
    n = args.npix
    p = t32(W.training_params(n, args.seed))
    syn = v.vfisv_synth(h, p, tf, tx, W.FE6173).reshape(n, 24)
    obs = (syn + 1e-3 * (p[:, 7] + p[:, 8])[:, None] * t32(W.noise(n, 24, args.seed))).contiguous()
    blob = v.vfisv_nn_init(h, obs, p, seed=args.seed)
    if args.train:
        v.vfisv_nn_train(h, blob, obs, p, batch=args.batch, epochs=1, lr0=1e-3, seed=2)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        loss = v.vfisv_nn_train(h, blob, obs, p, batch=args.batch, epochs=args.epochs, lr0=1e-3,
                                seed=3)
        e1.record()
        torch.cuda.synchronize()
        v.vfisv_check(h)
        ms = e0.elapsed_time(e1)
        steps = (n // args.batch) * args.epochs
        print(json.dumps({"npix": n, "batch": args.batch, "epochs": args.epochs, "steps": steps,
                          "ms": ms, "ms_per_step": ms / steps,
                          "tflops": FLOP_PER_TRAIN_SAMPLE * args.batch * steps / (ms / 1e3) / 1e12,
                          "loss_first": float(loss[:8].mean().item()),
                          "loss_last": float(loss[-8:].mean().item())}))
        h.close()
        return
    init = torch.empty((n, 10), dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        v.vfisv_nn_infer(h, blob, obs, W.FE6173, want_conf=False, init=init)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.iters):
        v.vfisv_nn_infer(h, blob, obs, W.FE6173, want_conf=False, init=init)
    e1.record()
    torch.cuda.synchronize()
    v.vfisv_check(h)
    ms = e0.elapsed_time(e1) / args.iters
    print(json.dumps({"npix": n, "ms": ms, "px_per_s": n / (ms * 1e-3),
                      "tflops": n * FLOP_PER_PIXEL / (ms * 1e-3) / 1e12,
                      "finite": bool(torch.isfinite(init).all().item())}))
    h.close()


if __name__ == "__main__":
    main()
