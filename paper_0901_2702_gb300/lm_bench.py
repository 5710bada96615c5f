"""One Levenberg-Marquardt inversion of a seeded synthetic map on the GPU:
the small, self-contained launch that profiles of the LM kernel capture.

The map has the uniform parameter distributions of the 1024x1024 workload
(B up to 3 kG, Fe I 6173 A, 6 filters x 149 wavelengths, noise 1e-3 Ic),
synthesised by the library itself.  Prints one JSON line with the time of
the timed inversion (CUDA events, after --warmup untimed ones).

    python -m paper_0901_2702_gb300.lm_bench --npix 262144 --no-cov [--fast-solve] [--autotune]
    python -m paper_0901_2702_gb300.lm_bench --npix 16384 --no-cov --tpp 2 --block 128
    python -m paper_0901_2702_gb300.lm_bench --npix 16384 --no-cov --spectrograph
"""
from __future__ import annotations

import argparse
import json
import os
import sys

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--npix", type=int, default=1 << 18)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-cov", action="store_true", help="skip the covariance output")
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--max-iter", type=int, default=50)
    ap.add_argument("--fast-solve", action="store_true", help="double-float solve (fast_solve=1)")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the pixel slots per CTA with vfisv_autotune first (as bench.py)")
    ap.add_argument("--tpp", type=int, default=0, help="threads per pixel (with --block)")
    ap.add_argument("--block", type=int, default=128, help="threads per CTA (with --tpp)")
    ap.add_argument("--spectrograph", action="store_true",
                    help="spectrograph-shaped inputs (112 samples x 4 Stokes, Fe I 6302.5 A)")
    args = ap.parse_args()

    import numpy as np
    import torch

    import paper_0901_2702_gb300 as v
    import workloads as W

    dev = torch.device("cuda:0")
    h = v.vfisv_create(0)
    t32 = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device=dev)  # noqa: E731
    if args.spectrograph:
        line = W.FE6302
        x, c = W.spectrograph_grid()
        tf, tx = t32(W.spectrograph_instrument(x, c)), t32(x)
    else:
        line = W.FE6173
        x = W.wavelength_grid()
        tf, tx = t32(W.hmi_filters(x)), t32(x)
    nobs = 4 * tf.shape[0]
    n = args.npix
    p = t32(W.quiet_and_active_params(n, args.seed))
    syn = v.vfisv_synth(h, p, tf, tx, line).reshape(n, nobs)
    sig = 1e-3 * (p[:, 7] + p[:, 8])[:, None]
    obs = (syn + sig * t32(W.noise(n, nobs, args.seed))).contiguous()
    w = (1.0 / (sig * sig)).expand(n, nobs).contiguous()
    cfg = {"max_iter": args.max_iter, "fast_solve": int(args.fast_solve)}
    block = tpp = None
    if args.tpp:
        v.vfisv_set_launch_shape(h, args.block, args.tpp)
        block, tpp = args.block, args.tpp
    if args.autotune:
        block, tpp, _ = v.vfisv_autotune(h, obs, w, tf, tx, line, config=cfg)
    for _ in range(args.warmup):
        v.vfisv_invert(h, obs, w, tf, tx, line, config=cfg, want_cov=not args.no_cov)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    r = v.vfisv_invert(h, obs, w, tf, tx, line, config=cfg, want_cov=not args.no_cov)
    e1.record()
    torch.cuda.synchronize()
    v.vfisv_check(h)
    st = r["status"]
    print(json.dumps({"npix": n, "ms": e0.elapsed_time(e1), "cov": not args.no_cov,
                      "fast_solve": bool(args.fast_solve), "spectrograph": args.spectrograph,
                      "lm_threads_per_cta": block, "lm_threads_per_pixel": tpp,
                      "mean_iters": r["iters"].float().mean().item(),
                      "passes": int(r["iters"].sum().item()) + n,
                      "converged": ((st == 0) | (st == 2)).float().mean().item()}))
    h.close()


if __name__ == "__main__":
    main()
