"""Run the oracle's per-pixel functions over chunks of pixels on all host
cores.  Every pixel is inverted independently, so the chunked result equals
one call over all pixels.  Worker processes are started with `spawn`: the
GPU tests call this after CUDA is initialised, and a forked child of a CUDA
process can hang.  Test infrastructure only (no method arithmetic here)."""
from __future__ import annotations

import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _init():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)


def _call(job):
    name, args, kw = job
    from oracle import lm
    return getattr(lm, name)(*args, **kw)


def workers(n_items: int, min_chunk: int = 16) -> int:
    return max(1, min(os.cpu_count() or 1, n_items // min_chunk))


def run(name: str, obs, w, *rest, chunk_args=(), procs: int | None = None, **kw):
    """oracle.lm.<name>(obs, w, *rest, **kw) over pixel chunks.  Arrays named
    in ``chunk_args`` (keyword names, e.g. ("init",)) are split with obs."""
    n = obs.shape[0]
    procs = procs or workers(n)
    if procs <= 1 or n < 2:
        return _call((name, (obs, w) + tuple(rest), kw))
    edges = np.linspace(0, n, procs + 1).astype(int)
    jobs = []
    for a, b in zip(edges[:-1], edges[1:]):
        k2 = dict(kw)
        for key in chunk_args:
            if kw.get(key) is not None:
                k2[key] = kw[key][a:b]
        jobs.append((name, (obs[a:b], w[a:b]) + tuple(rest), k2))
    ctx = mp.get_context("spawn")
    # one BLAS thread per worker (the workers already use every core)
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})
    try:
        with ctx.Pool(procs, initializer=_init) as pool:
            parts = pool.map(_call, jobs)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    out = {}
    for key in parts[0]:
        vals = [p_[key] for p_ in parts]
        if isinstance(vals[0], np.ndarray) and vals[0].ndim >= 1:
            out[key] = np.concatenate(vals)
        else:
            out[key] = vals
    return out
