"""Seeded synthetic inputs shaped like the VFISV workloads.

This module serves both the CUDA path and the FP64 oracle, so it holds none
of the inversion method's arithmetic: no Voigt/Faraday functions, no Zeeman
or Doppler constants, no radiative transfer, no chi-square.  It only draws
model parameters, noise and maps, and builds the wavelength grid and the
filter transmission tables, which are instrument data.

Workloads (all parameters in the C-ABI parameter order, see ``PARAM_NAMES``):

* ``quiet_and_active_params`` -- the uniform per-pixel distributions of the
  small and 1024x1024 plain-LM cases (B ~ U[0,3000] G, cos(gamma) ~ U[-1,1],
  psi ~ U[0,180) deg, eta0 ~ logU[1,50], Doppler width ~ U[20,50] mA,
  a ~ U[0,0.5], v ~ N(0,1.5) km/s clipped to +-7, S0 ~ U[0.1,0.4],
  S1 ~ U[0.6,0.9], alpha = 1).
* ``full_disk_params`` -- a 4096x4096 disk (radius 2073 px) with 90 % quiet
  Sun (B ~ U[0,200] G) and Gaussian active-region blobs (B up to 3500 G,
  smoothly varying inclination and azimuth).
* ``noise`` -- Gaussian noise of sigma = rel * I_c per observable, where the
  continuum I_c = S0 + mu*S1 of the generating model is passed in.
* ``serving_maps`` / ``serving_map_params`` -- the uneven serving mix: map
  sides log-uniform in [32, 2048], noise log-uniform in [3e-4, 3e-3] I_c,
  each map a disk with the full-disk distributions; half of the maps are
  spectrograph-shaped (``spectrograph_grid``, ``spectrograph_instrument``:
  112 samples 21.5 mA apart, Gaussian instrument FWHM 25 mA, synthesis grid
  4x finer, Fe I 6302.5 A).

The HMI-like instrument: 149 wavelength samples at 10 mA spacing over
+-740 mA about line centre (HMI tunes over the Fe I 6173 A line, paper
Sec. 1) and 6 filters centred at +-34.5, +-103.5, +-172.5 mA (69 mA spacing,
paper Sec. 4.1), each a Gaussian of FWHM 76 mA times a sinc^2 sidelobe
envelope, normalised to unit sum on the grid.
"""
from __future__ import annotations

import numpy as np

PARAM_NAMES = ("B", "gamma", "psi", "eta0", "dlambdaD", "a", "vlos", "S0", "S1", "alpha")
NPARAM = 10

# Fe I 6173 A line of the HMI workloads: lambda0 [A], effective Lande factor, mu.
FE6173 = {"lambda0_A": 6173.34, "geff": 2.5, "mu": 1.0}
# Fe I 6302.5 A (spectrograph-shaped inputs); lambda0 from the paper's Sec. 3.1.
FE6302 = {"lambda0_A": 6302.4936, "geff": 2.5, "mu": 1.0}

HMI_CENTRES_mA = (-172.5, -103.5, -34.5, 34.5, 103.5, 172.5)

SEEDS = {"small": 0, "map1024": 1, "disk": 2, "nn_train": 3, "nn_heldout": 4, "serving": 5}


def wavelength_grid(n: int = 149, step_mA: float = 10.0) -> np.ndarray:
    """Wavelength offsets from line centre in mA, symmetric about 0."""
    half = (n - 1) / 2.0
    return (np.arange(n, dtype=np.float64) - half) * step_mA


def hmi_filters(x_mA: np.ndarray, centres_mA=HMI_CENTRES_mA, fwhm_mA: float = 76.0,
                sidelobe_period_mA: float = 152.0) -> np.ndarray:
    """Filter transmission table [nfilt, nlam], each row summing to 1.

    T_k(x) = exp(-4 ln2 (x - c_k)^2 / FWHM^2) * sinc^2((x - c_k) / P), with
    sinc(t) = sin(pi t) / (pi t).
    """
    x = np.asarray(x_mA, dtype=np.float64)
    rows = []
    for c in centres_mA:
        d = x - c
        t = np.exp(-4.0 * np.log(2.0) * d * d / (fwhm_mA * fwhm_mA)) * np.sinc(d / sidelobe_period_mA) ** 2
        rows.append(t / t.sum())
    return np.stack(rows)


def gaussian_instrument(x_mA: np.ndarray, centres_mA, fwhm_mA: float) -> np.ndarray:
    """Gaussian instrument profiles [nfilt, nlam] (spectrograph-shaped inputs), unit sum."""
    x = np.asarray(x_mA, dtype=np.float64)
    rows = []
    for c in centres_mA:
        d = x - c
        t = np.exp(-4.0 * np.log(2.0) * d * d / (fwhm_mA * fwhm_mA))
        rows.append(t / t.sum())
    return np.stack(rows)


def _rng(seed: int, stream: int) -> np.random.Generator:
    # Philox is counter based; (seed, stream) selects an independent key.
    return np.random.Generator(np.random.Philox(key=[int(seed), int(stream)]))


def quiet_and_active_params(npix: int, seed: int, b_max: float = 3000.0) -> np.ndarray:
    """Per-pixel ME parameters [npix, 10] (float64) with the uniform distributions."""
    g = _rng(seed, 1)
    p = np.empty((npix, NPARAM), dtype=np.float64)
    p[:, 0] = g.uniform(0.0, b_max, npix)
    p[:, 1] = np.degrees(np.arccos(g.uniform(-1.0, 1.0, npix)))
    p[:, 2] = g.uniform(0.0, 180.0, npix)
    p[:, 3] = np.exp(g.uniform(np.log(1.0), np.log(50.0), npix))
    p[:, 4] = g.uniform(20.0, 50.0, npix)
    p[:, 5] = g.uniform(0.0, 0.5, npix)
    p[:, 6] = np.clip(g.normal(0.0, 1.5, npix), -7.0, 7.0)
    p[:, 7] = g.uniform(0.1, 0.4, npix)
    p[:, 8] = g.uniform(0.6, 0.9, npix)
    p[:, 9] = 1.0
    return p


def noise(npix: int, nobs: int, seed: int) -> np.ndarray:
    """Unit-variance Gaussian noise [npix, nobs] (float64)."""
    return _rng(seed, 2).standard_normal((npix, nobs))


def continuum(params: np.ndarray, mu: float = 1.0) -> np.ndarray:
    """Continuum level S0 + mu*S1 of the generating model, used to scale noise."""
    return params[:, 7] + mu * params[:, 8]


def observe(stokes: np.ndarray, params: np.ndarray, noise_unit: np.ndarray,
            sigma_rel: float = 1e-3, mu: float = 1.0):
    """Add noise of sigma = sigma_rel * I_c to stokes [npix, 4*nfilt].

    Returns (observed [npix, nobs], weights [npix, nobs]) with weights =
    w^2 / sigma^2 for w = 1.
    """
    ic = continuum(params, mu)[:, None]
    sig = sigma_rel * ic
    obs = stokes.reshape(stokes.shape[0], -1) + sig * noise_unit
    w = np.broadcast_to(1.0 / (sig * sig), obs.shape).copy()
    return obs, w


def disk_mask(side: int = 4096, radius: float = 2073.0) -> np.ndarray:
    c = (side - 1) / 2.0
    yy, xx = np.mgrid[0:side, 0:side]
    return (xx - c) ** 2 + (yy - c) ** 2 <= radius * radius


def disk_mu(idx: np.ndarray, side: int = 4096, radius: float = 2073.0) -> np.ndarray:
    """Heliocentric angle cosine mu = sqrt(1 - (r/R)^2) of flat pixel indices."""
    c = (side - 1) / 2.0
    x = (idx % side).astype(np.float64) - c
    y = (idx // side).astype(np.float64) - c
    return np.sqrt(np.clip(1.0 - (x * x + y * y) / (radius * radius), 0.0, 1.0))


def full_disk_params(seed: int, side: int = 4096, radius: float = 2073.0,
                     active_fraction: float = 0.10):
    """Full-disk map: returns (params [n_on_disk, 10], flat pixel indices).

    Quiet Sun pixels draw B ~ U[0,200] G and the other parameters as in
    ``quiet_and_active_params``.  Active regions are Gaussian blobs of FWHM
    ~ U[64,256] px with peak field ~ U[1500,3500] G, added until
    ``active_fraction`` of the on-disk pixels have blob weight > 0.5.  Inside
    a blob B = max(B_quiet, peak*weight), gamma = 90 - (90 - gamma_c)*weight
    with gamma_c in {0, 180}, and psi = radial angle about the blob centre.
    """
    mask = disk_mask(side, radius)
    idx = np.flatnonzero(mask)
    n = idx.size
    p = quiet_and_active_params(n, seed, b_max=200.0)
    g = _rng(seed, 3)
    c = (side - 1) / 2.0
    weight = np.zeros(side * side, dtype=np.float32)
    owner = np.full(side * side, -1, dtype=np.int32)
    blobs = []
    target = active_fraction * n
    covered = 0
    while covered < target:
        r = radius * np.sqrt(g.uniform(0.0, 0.9))
        th = g.uniform(0.0, 2.0 * np.pi)
        cx, cy = c + r * np.cos(th), c + r * np.sin(th)
        sig = g.uniform(64.0, 256.0) / 2.355
        peak = g.uniform(1500.0, 3500.0)
        gam_c = 0.0 if g.uniform() < 0.5 else 180.0
        k = len(blobs)
        blobs.append((cx, cy, sig, peak, gam_c))
        h = int(np.ceil(4 * sig))
        x0, x1 = max(0, int(cx) - h), min(side, int(cx) + h + 1)
        y0, y1 = max(0, int(cy) - h), min(side, int(cy) + h + 1)
        yy, xx = np.mgrid[y0:y1, x0:x1]
        wloc = np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * sig * sig)).astype(np.float32)
        flat = (yy * side + xx).ravel()
        wl = wloc.ravel()
        better = wl > weight[flat]
        weight[flat[better]] = wl[better]
        owner[flat[better]] = k
        covered = int(np.count_nonzero(weight[idx] > 0.5))
    w = weight[idx].astype(np.float64)
    own = owner[idx]
    act = own >= 0
    if act.any():
        bl = np.array(blobs)
        cx, cy, _, peak, gam_c = (bl[own[act], j] for j in range(5))
        px = (idx[act] % side).astype(np.float64)
        py = (idx[act] // side).astype(np.float64)
        wa = w[act]
        p[act, 0] = np.maximum(p[act, 0], peak * wa)
        p[act, 1] = 90.0 - (90.0 - gam_c) * wa
        p[act, 2] = np.mod(np.degrees(np.arctan2(py - cy, px - cx)), 180.0)
    return p, idx


def training_params(npix: int, seed: int) -> np.ndarray:
    """Training-set parameters for the initial-guess network (uniform draws)."""
    return quiet_and_active_params(npix, seed)


def serving_maps(seed: int, nmaps: int = 64, side_min: int = 32, side_max: int = 2048):
    """Side lengths and noise levels of the uneven batched serving mix."""
    g = _rng(seed, 4)
    sides = np.exp(g.uniform(np.log(side_min), np.log(side_max), nmaps)).astype(int)
    sig = np.exp(g.uniform(np.log(3e-4), np.log(3e-3), nmaps))
    return sides, sig


# Spectrograph-shaped inputs of the serving mix: the Fe I 6302.5 A line
# sampled at 112 points 21.5 mA apart, each sample a Gaussian instrument
# profile of FWHM 25 mA over a synthesis grid four times finer.
SPEC_NSAMP, SPEC_STEP_mA, SPEC_FINE = 112, 21.5, 4


def spectrograph_grid(nsamp: int = SPEC_NSAMP, step_mA: float = SPEC_STEP_mA,
                      fine: int = SPEC_FINE):
    """(fine synthesis grid [nsamp*fine], sample centres [nsamp]) in mA."""
    n = nsamp * fine
    x = (np.arange(n, dtype=np.float64) - (n - 1) / 2.0) * (step_mA / fine)
    c = (np.arange(nsamp, dtype=np.float64) - (nsamp - 1) / 2.0) * step_mA
    return x, c


def spectrograph_instrument(x_mA, centres_mA, fwhm_mA: float = 25.0, cut_fwhm: float = 3.0):
    """Gaussian instrument profiles [nsamp, nfine], truncated at cut_fwhm
    FWHM from each centre (tail mass < 1e-11), unit sum."""
    x = np.asarray(x_mA, dtype=np.float64)
    rows = []
    for c in centres_mA:
        d = x - c
        t = np.exp(-4.0 * np.log(2.0) * d * d / (fwhm_mA * fwhm_mA))
        t[np.abs(d) > cut_fwhm * fwhm_mA] = 0.0
        rows.append(t / t.sum())
    return np.stack(rows)


def serving_map_params(side: int, seed: int):
    """Parameters of one serving-mix map: a disk of diameter ~side with the
    full-disk distributions (quiet Sun and active-region blobs)."""
    side = max(int(side), 8)
    p, _ = full_disk_params(seed, side=side, radius=0.5 * side - 0.5,
                            active_fraction=0.10)
    return p
