"""A handle limited to a share of the SMs (vfisv_set_sm_limit) runs smaller
persistent grids; every per-pixel result depends on that pixel alone, so the
outputs equal those of the unlimited handle exactly."""
import numpy as np
import pytest

import workloads as W
from gpu_common import LINE, T, X, vf  # noqa: F401

pytestmark = pytest.mark.gpu


def _t32(torch, a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device=torch.device("cuda:0"))


def _equal(a, b):
    for k in a:
        if a[k] is not None:
            assert torch_equal(a[k], b[k]), k


def torch_equal(x, y):
    return bool((x == y).all().item()) if hasattr(x, "device") else np.array_equal(x, y)


@pytest.mark.parametrize("nsm", [1, 19, 100])
def test_sm_limit_keeps_results(vf, nsm):
    v, h, torch = vf
    n = 30000
    tf, tx = _t32(torch, T), _t32(torch, X)
    p = _t32(torch, W.quiet_and_active_params(n, 81))
    syn = v.vfisv_synth(h, p, tf, tx, LINE).reshape(n, 24)
    sig = 1e-3 * (p[:, 7] + p[:, 8])[:, None]
    obs = (syn + sig * _t32(torch, W.noise(n, 24, 81))).contiguous()
    w = (1.0 / (sig * sig)).expand(n, 24).contiguous()
    blob = v.vfisv_nn_init(h, obs, p, seed=5)
    r0 = v.vfisv_invert(h, obs, w, tf, tx, LINE, config={"max_iter": 30}, want_cov=True)
    g0 = v.vfisv_nn_infer(h, blob, obs, LINE, want_raw=True)
    v.vfisv_set_sm_limit(h, nsm)
    try:
        r1 = v.vfisv_invert(h, obs, w, tf, tx, LINE, config={"max_iter": 30}, want_cov=True)
        g1 = v.vfisv_nn_infer(h, blob, obs, LINE, want_raw=True)
    finally:
        v.vfisv_set_sm_limit(h, 0)
    _equal(r0, r1)
    _equal(g0, g1)
    v.vfisv_check(h)


def test_sm_limit_spectrograph_path(vf):
    v, h, torch = vf
    x, c = W.spectrograph_grid()
    F = W.spectrograph_instrument(x, c)
    tf, tx = _t32(torch, F), _t32(torch, x)
    n = 2000
    p = _t32(torch, W.quiet_and_active_params(n, 82))
    syn = v.vfisv_synth(h, p, tf, tx, W.FE6302).reshape(n, -1)
    obs = (syn + 1e-3 * _t32(torch, W.noise(n, syn.shape[1], 82))).contiguous()
    w = torch.full((syn.shape[1],), 1e6, device=obs.device)
    cfg = {"max_iter": 20, "wfa_pol": 1.0}
    r0 = v.vfisv_invert(h, obs, w, tf, tx, W.FE6302, config=cfg, want_cov=True)
    v.vfisv_set_sm_limit(h, 7)
    try:
        r1 = v.vfisv_invert(h, obs, w, tf, tx, W.FE6302, config=cfg, want_cov=True)
    finally:
        v.vfisv_set_sm_limit(h, 0)
    _equal(r0, r1)
    with pytest.raises(v.VfisvError):
        v.vfisv_set_sm_limit(h, -1)
    v.vfisv_check(h)
