"""Many maps in one launch (vfisv_invert_batch): the same results as one
vfisv_invert call per map with that map's weights (the arithmetic of a pixel
does not depend on its neighbours), per-map latencies that are ordered and
bounded by the call, and parity with the oracle per map."""
import time

import numpy as np
import pytest

import workloads as W
from oracle import lm
from gpu_common import LINE, T, X, f32, vf  # noqa: F401

pytestmark = pytest.mark.gpu


def _maps(v, h, torch, instrument, sizes, seed):
    dev = torch.device("cuda:0")
    if instrument == "filter":
        x, F, line = X, T, LINE
    else:
        x, c = W.spectrograph_grid()
        F, line = W.spectrograph_instrument(x, c), W.FE6302
    t32 = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device=dev)  # noqa: E731
    tf, tx = t32(F), t32(x)
    obs, wts = [], []
    for m, n in enumerate(sizes):
        p = t32(W.quiet_and_active_params(max(n, 1), seed + m))[:n]
        sig = 3e-4 * (10 ** (m % 2))
        if n:
            s = v.vfisv_synth(h, p, tf, tx, line).reshape(n, -1)
            obs.append(s + sig * t32(W.noise(n, s.shape[1], seed + m)))
        wts.append(torch.full((4 * F.shape[0],), 1.0 / sig ** 2, device=dev))
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return torch.cat(obs).contiguous(), torch.stack(wts).contiguous(), off, tf, tx, line


@pytest.mark.parametrize("instrument,sizes", [("filter", [700, 0, 1300, 45]),
                                              ("spectrograph", [96, 160])])
def test_batch_equals_per_map_calls(vf, instrument, sizes):
    v, h, torch = vf
    obs, wts, off, tf, tx, line = _maps(v, h, torch, instrument, sizes, 110)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b = v.vfisv_invert_batch(h, obs, wts, off, tf, tx, line)
    v.vfisv_check(h)
    wall_ms = (time.perf_counter() - t0) * 1e3
    lat = b["latency_ms"].cpu().numpy()
    for m in range(len(sizes)):
        lo, hi = off[m], off[m + 1]
        if hi == lo:
            assert lat[m] == 0.0
            continue
        r = v.vfisv_invert(h, obs[lo:hi].contiguous(), wts[m].contiguous(), tf, tx, line)
        v.vfisv_check(h)
        for k in ("params", "chi2", "iters", "status", "cov"):
            assert torch.equal(b[k][lo:hi], r[k]), (m, k)
        assert 0.0 < lat[m] <= wall_ms
    print(f"{instrument}: latencies {np.round(lat, 3)} ms, call {wall_ms:.2f} ms")


def test_batch_vs_oracle(vf):
    v, h, torch = vf
    sizes = [150, 250]
    obs, wts, off, tf, tx, line = _maps(v, h, torch, "filter", sizes, 120)
    b = v.vfisv_invert_batch(h, obs, wts, off, tf, tx, line)
    v.vfisv_check(h)
    o_all = f32(obs.cpu().numpy())
    for m in range(2):
        lo, hi = off[m], off[m + 1]
        w = np.broadcast_to(f32(wts[m].cpu().numpy()), (hi - lo, 24))
        o = lm.invert(o_all[lo:hi], w, f32(T), f32(X), LINE)
        g = {k: b[k][lo:hi].cpu().numpy() for k in ("chi2", "status")}
        both = np.isin(g["status"], (0, 2)) & np.isin(o["status"], (0, 2))
        rel = np.abs(g["chi2"][both] / o["chi2"][both] - 1)
        assert both.mean() > 0.5 and np.mean(rel <= 1e-3) >= 0.97
