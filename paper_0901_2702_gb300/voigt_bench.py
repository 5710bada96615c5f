"""Voigt / Faraday-Voigt evaluation speed on the GPU (the paper's Sec. 3.2
timing experiment, Fig. 3): the Weideman rational series vs first- and
second-order Taylor extrapolation from the 500 x 100 table, for growing
numbers of points.  Prints one JSON line per (method, n).

    python -m paper_0901_2702_gb300.voigt_bench
"""
from __future__ import annotations

import json
import os
import sys

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    import torch

    import paper_0901_2702_gb300 as v
    dev = torch.device("cuda:0")
    h = v.vfisv_create(0)
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    nmax = 1 << 26
    # dampings and frequencies spanning a typical inversion (a < 0.5, |u| < 20)
    a = torch.rand(nmax, device=dev, generator=g) * 0.5
    u = (torch.rand(nmax, device=dev, generator=g) * 2 - 1) * 20
    names = {0: "rational (Weideman, 16 terms)", 1: "Taylor table, 1st order",
             2: "Taylor table, 2nd order"}
    for method in (0, 1, 2):
        for n in (10_000, 100_000, 1_000_000, 10_000_000, nmax):
            aa, uu = a[:n], u[:n]
            for _ in range(3):
                v.vfisv_voigt(h, aa, uu, method)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            reps = max(1, min(200, int(2e8 // n)))
            e0.record()
            for _ in range(reps):
                v.vfisv_voigt(h, aa, uu, method)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            print(json.dumps({"method": names[method], "n": n, "ms": ms,
                              "evaluations_per_s": n / (ms / 1e3)}))
    h.close()


if __name__ == "__main__":
    main()
