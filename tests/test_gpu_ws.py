"""The warp-specialised LM kernel (launch shape 384 x 1: a producer warpgroup
running the fused wavelength pass, two consumer warpgroups running chi2,
the normal equations and the FP64 solve, the filtered rows handed over in
tensor memory) against the one-warpgroup kernel (128 x 1).  Both run the
same passes, decisions and sums in the same order, so every output must
agree bit for bit; parity with the oracle then carries over from the tests
of the 128 x 1 kernel.  Cases: a map with more pixels than the resident
slots (152 SMs x 256) so slots refill from the queue, tiny maps that leave
most slots and whole consumer warps idle, initial models, Hessian reuse,
an iteration cap of 0 and 1, bad input pixels, the work counters, a handle
limited to fewer SMs, graph replay, batched maps, the mixed inversion
with confidence routing (pixel list and device-side count), and wavelength
grids of 37 and 4096 points (the largest filter table the library takes),
with a direct oracle comparison on the coarse grid."""
import numpy as np
import pytest

import workloads as W
from gpu_common import LINE, T, X, f32, vf  # noqa: F401

pytestmark = pytest.mark.gpu


def _map(v, h, torch, n, seed, bad=(), T_=T, X_=X):
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(np.asarray(a, np.float32), device=dev)  # noqa: E731
    p = W.quiet_and_active_params(n, seed)
    tf, tx = t(T_), t(X_)
    syn = v.vfisv_synth(h, t(p), tf, tx, LINE).reshape(n, 24)
    sig = 1e-3 * t(W.continuum(p))[:, None]
    obs = (syn + sig * t(W.noise(n, 24, seed))).contiguous()
    w = (1.0 / (sig * sig)).expand(n, 24).contiguous()
    for i in bad:
        obs[i, 3] = float("nan")
    torch.cuda.synchronize()
    return p, obs, w, tf, tx


def _both(v, h, obs, w, tf, tx, **kw):
    out = []
    for block in (128, 384):
        v.vfisv_set_launch_shape(h, block, 1)
        try:
            v.vfisv_counters(h, reset=True)
            r = v.vfisv_invert(h, obs, w, tf, tx, LINE, **kw)
            v.vfisv_check(h)
            out.append((r, v.vfisv_counters(h, reset=True)))
        finally:
            v.vfisv_set_launch_shape(h, 128, 1)
    return out


def _same(torch, a, b):
    for k in a:
        if a[k] is None:
            assert b[k] is None
            continue
        assert torch.equal(a[k], b[k]), k


@pytest.mark.parametrize("n", [1, 37, 300, 40077])
def test_same_results_as_one_warpgroup_kernel(vf, n):
    v, h, torch = vf
    p, obs, w, tf, tx = _map(v, h, torch, n, 500 + n, bad=(0,) if n > 1 else ())
    (a, ca), (b, cb) = _both(v, h, obs, w, tf, tx)
    _same(torch, a, b)
    assert ca == cb, (ca, cb)
    assert cb["retired"] == n - (1 if n > 1 else 0)
    if n > 1:
        assert int(b["status"][0]) == 3  # the NaN pixel: bad input


def test_same_results_with_initial_models_and_options(vf):
    v, h, torch = vf
    n = 5000
    p, obs, w, tf, tx = _map(v, h, torch, n, 77)
    init = torch.tensor(np.asarray(p, np.float32), device="cuda:0")
    init[:, 0] *= 1.2
    init[:, 3] *= 0.8
    for cfg in ({"max_iter": 20}, {"hess_reuse": 1e-2}, {"max_iter": 0}, {"max_iter": 1}):
        (a, ca), (b, cb) = _both(v, h, obs, w, tf, tx, init=init, config=cfg)
        _same(torch, a, b)
        assert ca == cb, (cfg, ca, cb)
    (a, _), (b, _) = _both(v, h, obs, w, tf, tx, want_cov=False)
    _same(torch, a, b)


def test_configurations_it_does_not_take_fall_back(vf):
    """fast_solve and restarts run the one-warpgroup kernel whatever the shape."""
    v, h, torch = vf
    p, obs, w, tf, tx = _map(v, h, torch, 2000, 91)
    for cfg in ({"fast_solve": 1}, {"restarts": 1, "seed": 77, "max_iter": 30}):
        (a, _), (b, _) = _both(v, h, obs, w, tf, tx, config=cfg)
        _same(torch, a, b)


def test_sm_limit_and_graph_replay(vf):
    """Execution-only changes with the warp-specialised shape: a handle
    limited to 19 SMs (fewer CTAs, the same queue) and a captured graph
    replayed on new observations give the unlimited direct call's results
    bit for bit."""
    v, h, torch = vf
    n = 20000
    p, obs, w, tf, tx = _map(v, h, torch, n, 71)
    _, obs2, _, _, _ = _map(v, h, torch, n, 72)
    v.vfisv_set_launch_shape(h, 384, 1)
    try:
        ref = v.vfisv_invert(h, obs, w, tf, tx, LINE)
        v.vfisv_set_sm_limit(h, 19)
        try:
            lim = v.vfisv_invert(h, obs, w, tf, tx, LINE)
            v.vfisv_check(h)
        finally:
            v.vfisv_set_sm_limit(h, 0)
        _same(torch, ref, lim)
        dev = torch.device("cuda:0")
        s = torch.cuda.Stream(dev)
        out = {k: torch.empty_like(t_) for k, t_ in ref.items()}
        src = obs.clone()
        with torch.cuda.stream(s):
            v.vfisv_invert(h, src, w, tf, tx, LINE, out=out, stream=s)  # sizes the workspaces
            s.synchronize()
            v.vfisv_graph_begin(h, s)
            v.vfisv_invert(h, src, w, tf, tx, LINE, out=out, stream=s)
            g = v.vfisv_graph_end(h, s)
            for data in (obs, obs2):
                src.copy_(data)
                g.launch(s)
                s.synchronize()
                direct = v.vfisv_invert(h, data, w, tf, tx, LINE, stream=s)
                s.synchronize()
                _same(torch, out, direct)
        g.close()
        v.vfisv_check(h)
    finally:
        v.vfisv_set_launch_shape(h, 128, 1)


def test_batched_maps_same_results(vf):
    """Many maps in one launch (vfisv_invert_batch, per-map weights and
    completion stamps) with the warp-specialised shape: the per-pixel outputs
    equal the one-warpgroup kernel's bit for bit, every map gets a stamp."""
    v, h, torch = vf
    sizes = [1, 700, 33, 5000, 129]
    parts = [_map(v, h, torch, n, 900 + i) for i, n in enumerate(sizes)]
    obs = torch.cat([q[1] for q in parts]).contiguous()
    w = torch.stack([q[2][0] * (1.0 + 0.1 * i) for i, q in enumerate(parts)]).contiguous()
    tf, tx = parts[0][3], parts[0][4]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    res = []
    for block in (128, 384):
        v.vfisv_set_launch_shape(h, block, 1)
        try:
            r = v.vfisv_invert_batch(h, obs, w, off, tf, tx, LINE)
            v.vfisv_check(h)
            res.append(r)
        finally:
            v.vfisv_set_launch_shape(h, 128, 1)
    a, b = res
    for k in a:
        if k == "latency_ms":
            assert bool((b[k] > 0).all()), b[k]
            continue
        assert torch.equal(a[k], b[k]), k


def test_mixed_inversion_with_routing_same_results(vf):
    """The mixed inversion (network guess, confidence routing to plain LM
    through the LM kernel's device-side pixel list and count, flagged pixels
    re-inverted, one covariance pass over the merged rows) with the
    warp-specialised shape equals the one-warpgroup kernel's bit for bit.
    An untrained network serves: only the equality of the two shapes is
    tested, whatever it routes."""
    v, h, torch = vf
    n = 6000
    p, obs, w, tf, tx = _map(v, h, torch, n, 131)
    blob = v.vfisv_nn_init(h, obs, torch.tensor(np.asarray(p, np.float32), device="cuda:0"),
                           seed=5)
    conf = v.vfisv_nn_infer(h, blob, obs, LINE)["conf"]
    k = float(conf.median().item())  # about half the pixels routed
    res = []
    for block in (128, 384):
        v.vfisv_set_launch_shape(h, block, 1)
        try:
            r = v.vfisv_invert_nn(h, blob, obs, w, tf, tx, LINE, config_nn={"max_iter": 20},
                                  config_plain={"max_iter": 50}, chi2_flag=3.0,
                                  flag_unconverged=True, conf_route=k)
            v.vfisv_check(h)
            res.append(r)
        finally:
            v.vfisv_set_launch_shape(h, 128, 1)
    a, b = res
    assert 0.2 < float((conf > k).float().mean().item()) < 0.8
    for key in a:
        if a[key] is None:
            continue
        assert torch.equal(a[key], b[key]), key


def _grid(nlam):
    x = np.linspace(-600.0, 650.0, nlam)
    return x, W.hmi_filters(x)


@pytest.mark.parametrize("nlam", [37, 4096])
def test_same_results_on_other_grids(vf, nlam):
    """A coarse 37-point grid and the largest grid the library takes (4096
    points: the filter table then fills most of the shared memory of both
    kernels)."""
    v, h, torch = vf
    x, Tg = _grid(nlam)
    n = 3000
    p, obs, w, tf, tx = _map(v, h, torch, n, 600 + nlam, T_=Tg, X_=x)
    (a, ca), (b, cb) = _both(v, h, obs, w, tf, tx)
    _same(torch, a, b)
    assert ca == cb, (ca, cb)
    assert cb["retired"] == n


def test_oracle_parity_on_a_coarse_grid(vf):
    """The warp-specialised kernel against the FP64 oracle on the 37-point
    grid (observations synthesised by the oracle, every input rounded to
    float32 first): chi2 within 1e-3 for >= 98 % of the pixels converged in
    both, the bar of the 149-point parity tests."""
    from oracle import lm, me
    v, h, torch = vf
    x, Tg = _grid(37)
    n = 300
    p = f32(W.quiet_and_active_params(n, 611))
    s = me.synth(p, f32(Tg), f32(x), LINE).reshape(n, -1)
    obs, w = W.observe(s, p, W.noise(n, 24, 611))
    obs, w = f32(obs), f32(w)
    t = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda:0")  # noqa: E731
    v.vfisv_set_launch_shape(h, 384, 1)
    try:
        r = v.vfisv_invert(h, t(obs), t(w), t(Tg), t(x), LINE)
        v.vfisv_check(h)
    finally:
        v.vfisv_set_launch_shape(h, 128, 1)
    g = {k: a.cpu().numpy() for k, a in r.items() if a is not None}
    o = lm.invert(obs, w, f32(Tg), f32(x), LINE)
    both = np.isin(g["status"], (0, 2)) & np.isin(o["status"], (0, 2))
    rel = np.abs(g["chi2"] / np.where(o["chi2"] > 0, o["chi2"], 1) - 1)
    assert both.mean() > 0.4, both.mean()
    assert np.mean(rel[both] <= 1e-3) >= 0.98, np.sort(rel[both])[-10:]
