"""GPU synthesis vs the FP64 oracle: |S_gpu - S_oracle| <= 1e-5 Ic per
observable (Ic = S0 + mu S1 of the pixel), on the small 64x64 workload,
edge cases, every compiled filter count, ragged sizes, and a sample of the
1024x1024 map synthesised in one launch."""
import numpy as np
import pytest

import workloads as W
from oracle import me
from gpu_common import LINE, T, X, f32, vf  # noqa: F401

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _gpu(v, h, torch, p, T_=T, x_=X, line=LINE):
    dev = torch.device("cuda:0")
    out = v.vfisv_synth(h, torch.tensor(p, dtype=torch.float32, device=dev),
                        torch.tensor(T_, dtype=torch.float32, device=dev),
                        torch.tensor(x_, dtype=torch.float32, device=dev), line)
    v.vfisv_check(h)
    return out.cpu().numpy().astype(np.float64)


def _err(gpu, ref, p):
    ic = (p[:, 7] + p[:, 8])[:, None, None]
    return np.abs(gpu - ref) / ic


def test_small_workload_parity(vf):
    v, h, torch = vf
    p = f32(W.quiet_and_active_params(4096, W.SEEDS["small"]))
    e = _err(_gpu(v, h, torch, p), me.synth(p, f32(T), f32(X), LINE), p)
    assert e.max() <= TOL, e.max()


def test_special_cases_exact(vf):
    v, h, torch = vf
    p = f32(W.quiet_and_active_params(64, 3))
    p[:32, 0] = 0.0          # no field: no polarisation
    p[32:, 1] = 0.0          # longitudinal field: no linear polarisation
    g = _gpu(v, h, torch, p)
    assert np.all(g[:32, 1:] == 0.0)
    assert np.all(g[32:, 1:3] == 0.0)


def test_filling_factor_and_extremes(vf):
    v, h, torch = vf
    p = f32(W.quiet_and_active_params(256, 4))
    p[:, 9] = np.linspace(0.0, 1.0, 256)
    p[:16, 0] = 6000.0; p[16:32, 3] = 500.0; p[32:48, 3] = 0.01; p[48:64, 4] = 5.0
    p[64:80, 4] = 150.0; p[80:96, 5] = 5.0; p[96:112, 5] = 0.0; p[112:128, 6] = 20.0
    p = f32(p)
    e = _err(_gpu(v, h, torch, p), me.synth(p, f32(T), f32(X), LINE), p)
    assert e.max() <= TOL, e.max()


@pytest.mark.parametrize("nf", [1, 2, 3, 4, 5, 6, 7, 8])
def test_every_filter_count(vf, nf):
    v, h, torch = vf
    cent = np.linspace(-200, 200, nf)
    Tn = W.hmi_filters(X, centres_mA=cent)
    p = f32(W.quiet_and_active_params(333, 5 + nf))
    e = _err(_gpu(v, h, torch, p, T_=Tn), me.synth(p, f32(Tn), f32(X), LINE), p)
    assert e.max() <= TOL, (nf, e.max())


@pytest.mark.parametrize("nlam", [1, 37, 1000])
def test_ragged_grids(vf, nlam):
    v, h, torch = vf
    x = np.linspace(-600, 650, nlam) if nlam > 1 else np.array([12.5])
    Tn = W.hmi_filters(x) if nlam > 1 else np.ones((6, 1))
    p = f32(W.quiet_and_active_params(129, 9))
    e = _err(_gpu(v, h, torch, p, T_=Tn, x_=x), me.synth(p, f32(Tn), f32(x), LINE), p)
    assert e.max() <= TOL, (nlam, e.max())


def test_empty_and_host_buffers(vf):
    v, h, torch = vf
    p = f32(W.quiet_and_active_params(77, 10))
    dev = v.vfisv_synth(h, torch.tensor(p, dtype=torch.float32, device="cuda:0"),
                        torch.tensor(T, dtype=torch.float32, device="cuda:0"),
                        torch.tensor(X, dtype=torch.float32, device="cuda:0"), LINE)
    host = v.vfisv_synth(h, p.astype(np.float32), T.astype(np.float32), X.astype(np.float32), LINE)
    assert np.array_equal(dev.cpu().numpy(), host)
    empty = v.vfisv_synth(h, np.zeros((0, 10), np.float32), T.astype(np.float32),
                          X.astype(np.float32), LINE)
    assert empty.shape == (0, 4, 6)


def test_other_lines(vf):
    v, h, torch = vf
    p = f32(W.quiet_and_active_params(128, 11))
    for line in (W.FE6302, {"lambda0_A": 15648.515, "geff": 3.0, "mu": 0.6}):
        e = _err(_gpu(v, h, torch, p, line=line), me.synth(p, f32(T), f32(X), line), p)
        assert e.max() <= TOL, (line, e.max())


def test_full_map_sampled(vf):
    """1024x1024 parameters synthesised in one launch; 2048 sampled pixels vs the oracle."""
    v, h, torch = vf
    npix = 1024 * 1024
    p = f32(W.quiet_and_active_params(npix, W.SEEDS["map1024"]))
    g = _gpu(v, h, torch, p)
    idx = np.random.default_rng(0).choice(npix, 2048, replace=False)
    e = _err(g[idx], me.synth(p[idx], f32(T), f32(X), LINE), p[idx])
    assert e.max() <= TOL, e.max()


def _kept_rows(T_):
    """The grid points the packed table keeps (host restatement of the packing
    rule): the points of least relative weight max_k |T_k| / sum |T_k| are
    dropped while every filter's dropped |weights| stay within 2^-24 of its
    total."""
    A = np.abs(T_).astype(np.float64)
    M = A.sum(axis=1)
    r = (A / M[:, None]).max(axis=0)
    order = np.argsort(r, kind="stable")
    within = (np.cumsum(A[:, order], axis=1) <= 2.0 ** -24 * M[:, None]).all(axis=0)
    ndrop = len(order) if within.all() else int(np.argmin(within))
    keep = np.ones(A.shape[1], dtype=bool)
    keep[order[:ndrop]] = False
    return keep


def test_negligible_grid_points_left_out(vf):
    """The packed table leaves out the grid points that carry, together, at
    most 2^-24 of every filter's weight (for the HMI-like filters on the
    149-point grid: the wings beyond +-310 mA, 86 of 149 points).  Synthesis
    through the full grid and through a grid the caller has already cut to
    the kept points agree to FP32 rounding (the cut grid may drop a few more
    points under the same rule, and tau, summed over every point, may move
    by an ulp), and both stay within the parity bound of the oracle's
    full-grid sums."""
    v, h, torch = vf
    keep = _kept_rows(f32(T))
    assert keep.sum() == 63 and np.flatnonzero(keep)[[0, -1]].tolist() == [43, 105]
    p = f32(W.quiet_and_active_params(2048, 55))
    full = _gpu(v, h, torch, p)
    cut = _gpu(v, h, torch, p, T_=T[:, keep], x_=X[keep])
    ic = (p[:, 7] + p[:, 8])[:, None, None]
    assert (np.abs(full - cut) / ic).max() <= 2e-7
    ref = me.synth(p, f32(T), f32(X), LINE)
    assert _err(full, ref, p).max() <= TOL
    # a filter table without negligible points keeps every point
    T2 = np.full((6, 37), 1.0 / 37)
    x2 = np.linspace(-200, 200, 37)
    e = _err(_gpu(v, h, torch, p[:64], T_=T2, x_=x2), me.synth(p[:64], f32(T2), f32(x2), LINE),
             p[:64])
    assert e.max() <= TOL
