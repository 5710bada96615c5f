"""Host buffers on a large map take the library's copy/compute pipeline
(chunks copied in and out on their own streams while the previous chunk is
inverted).  Every per-pixel result depends on that pixel alone, so the
pipelined call must reproduce the call on device buffers exactly."""
import numpy as np
import pytest

import workloads as W
from gpu_common import LINE, T, X, vf  # noqa: F401

pytestmark = pytest.mark.gpu

# above the library's pipeline threshold (2^20 pixels), ragged last chunk
NPIX = (1 << 20) + 12345


def _map(v, h, torch, seed):
    dev = torch.device("cuda:0")
    t32 = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device=dev)  # noqa: E731
    tf, tx = t32(T), t32(X)
    p = t32(W.quiet_and_active_params(NPIX, seed))
    syn = v.vfisv_synth(h, p, tf, tx, LINE).reshape(NPIX, 24)
    sig = 1e-3 * (p[:, 7] + p[:, 8])[:, None]
    obs = (syn + sig * t32(W.noise(NPIX, 24, seed))).contiguous()
    w = (1.0 / (sig * sig)).expand(NPIX, 24).contiguous()
    return obs, w, tf, tx, p


def _host(t):
    return t.cpu().numpy().copy()


def _same(host, dev):
    for k, a in host.items():
        if a is None:
            continue
        np.testing.assert_array_equal(a, dev[k].cpu().numpy(), err_msg=k)


@pytest.mark.parametrize("chunks", [2, 3, 5])
def test_plain_inversion_host_pipeline(vf, chunks):
    """2 chunks: equal halves; 3 (the default) and 5: small first and last."""
    v, h, torch = vf
    obs, w, tf, tx, _ = _map(v, h, torch, 71)
    cfg = {"max_iter": 30}
    rd = v.vfisv_invert(h, obs, w, tf, tx, LINE, config=cfg, want_cov=True)
    v.vfisv_set_pipeline_chunks(h, chunks)
    try:
        rh = v.vfisv_invert(h, _host(obs), _host(w), _host(tf), _host(tx), LINE, config=cfg,
                            want_cov=True)
    finally:
        v.vfisv_set_pipeline_chunks(h, 3)
    assert isinstance(rh["params"], np.ndarray)
    _same(rh, rd)
    v.vfisv_check(h)


def test_pipeline_depth_bounds(vf):
    v, h, torch = vf
    for bad in (-1, 65):
        with pytest.raises(v.VfisvError):
            v.vfisv_set_pipeline_chunks(h, bad)
    v.vfisv_set_pipeline_chunks(h, 3)


@pytest.mark.parametrize("route", [False, True])
def test_mixed_inversion_host_pipeline(vf, route):
    v, h, torch = vf
    obs, w, tf, tx, p = _map(v, h, torch, 72)
    blob = v.vfisv_nn_init(h, obs, p, seed=3)
    k = float(v.vfisv_nn_infer(h, blob, obs, LINE)["conf"].median().item()) if route \
        else float("inf")
    kw = dict(config_nn={"max_iter": 20}, config_plain={"max_iter": 30}, chi2_flag=2.5,
              conf_route=k, want_cov=True)
    rd = v.vfisv_invert_nn(h, blob, obs, w[0].contiguous(), tf, tx, LINE, **kw)
    rh = v.vfisv_invert_nn(h, _host(blob), _host(obs), _host(w[0]), _host(tf), _host(tx), LINE,
                           **kw)
    _same(rh, rd)
    v.vfisv_check(h)
