"""vfisv_invert_noalloc, the inversion entry point for callers that may not
allocate device memory (a host framework that owns every byte through its
own pool, or a real-time pipeline that allocates only at start-up because
cudaMalloc/cudaFree can synchronise the device).  It keeps its scratch in a
fixed array inside the library.  Called twice in a row, on two different
maps, through the C ABI, it must reproduce the handle-based vfisv_invert;
so must a map larger than the array's resident pixel slots (60,000 pixels
against VFISV_NOALLOC_MAX_SLOTS = 38,912: the slots refill from the work
queue, and where the GPU could hold more slots than the array the grid is
capped) and the double-float solve option.  vfisv_noalloc_check, its
error-word companion, reports no device error after each call.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _map(v, h, torch, n, seed):
    dev = torch.device("cuda:0")
    x = W.wavelength_grid()
    T = W.hmi_filters(x)
    p = W.quiet_and_active_params(n, seed)
    t = lambda a: torch.tensor(a, dtype=torch.float32, device=dev)  # noqa: E731
    tf, tx, tp = t(T), t(x), t(p)
    syn = v.vfisv_synth(h, tp, tf, tx, W.FE6173).reshape(n, 24)
    sig = 1e-3 * (tp[:, 7] + tp[:, 8])[:, None]
    obs = (syn + sig * t(W.noise(n, 24, seed))).contiguous()
    w = (1.0 / (sig * sig)).expand(n, 24).contiguous()
    return obs, w, tf, tx


def _noalloc(v, torch, obs, w, tf, tx, cfg):
    lib = v.load()
    f = lib.vfisv_invert_noalloc
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    f.argtypes = [P, P, I32, P, I32, P, I32, ctypes.POINTER(v.vfisv_line), P,
                  ctypes.POINTER(v.vfisv_config), I64, P, P, P, P, P, P]
    f.restype = ctypes.c_int
    n = obs.shape[0]
    dev = obs.device
    out = {"params": torch.empty(n, 10, device=dev), "chi2": torch.empty(n, device=dev),
           "iters": torch.empty(n, dtype=torch.int32, device=dev),
           "status": torch.empty(n, dtype=torch.int32, device=dev),
           "cov": torch.empty(n, 10, 10, device=dev)}
    line = v._line(W.FE6173)
    rc = f(obs.data_ptr(), w.data_ptr(), 1, tf.data_ptr(), tf.shape[0], tx.data_ptr(),
           tf.shape[1], ctypes.byref(line), None, ctypes.byref(cfg), n,
           out["params"].data_ptr(), out["chi2"].data_ptr(), out["iters"].data_ptr(),
           out["status"].data_ptr(), out["cov"].data_ptr(),
           ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
    assert rc == 0, v.vfisv_strerror(rc)
    chk = lib.vfisv_noalloc_check
    chk.argtypes = [P]
    chk.restype = ctypes.c_int
    rc = chk(ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
    assert rc == 0, v.vfisv_strerror(rc)
    torch.cuda.synchronize()
    return {k: t.cpu().numpy() for k, t in out.items()}


def test_noalloc_matches_handle_path_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0901_2702_gb300 import build
    build.build()
    import paper_0901_2702_gb300 as v
    h = v.vfisv_create(0)
    # two different maps, one call each, back to back on the shared array;
    # then a map with more pixels than resident slots, and the double-float
    # solve
    for n, seed, fast in ((3000, 21, 0), (1100, 22, 0), (60000, 23, 0), (5000, 24, 1)):
        cfg = v.vfisv_config_default(fast_solve=fast)
        obs, w, tf, tx = _map(v, h, torch, n, seed)
        got = _noalloc(v, torch, obs, w, tf, tx, cfg)
        ref = v.vfisv_invert(h, obs, w, tf, tx, W.FE6173, config=cfg)
        v.vfisv_check(h)
        ref = {k: t.cpu().numpy() for k, t in ref.items()}
        assert np.array_equal(got["status"], ref["status"])
        assert np.array_equal(got["iters"], ref["iters"])
        for k in ("params", "chi2", "cov"):
            np.testing.assert_allclose(got[k], ref[k], rtol=1e-6, atol=1e-12)
    h.close()
