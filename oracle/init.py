"""Initial models from the observed filtergrams (Sec. 5), FP64 (oracle).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

The paper initialises B and gamma with a magnetograph / weak-field
estimate (after Jefferies & Mickey 1991) when the polarisation is below
6 %, with the network above, and the azimuth always with the method of
Auer et al. (1977); neither method is spelled out.  Read here as the
weak-field relations between the Stokes samples and the wavelength
derivatives of Stokes I, evaluated on the filtergrams themselves:

* filter centres c_k = sum_i T_k(x_i) x_i / sum_i T_k(x_i), filters taken in
  increasing c_k;
* first derivative of I across the centres: central differences inside,
  one-sided at the two ends; second derivative at the interior centres
  from the two adjacent slopes;
* longitudinal field: V_k = s_V C B_par dI/dlambda_k fitted by least
  squares, C = 4.66685e-10 g lambda0^2 mA/G (Eq. 7);
* transverse field: |(Q_k, U_k)| = C^2 B_perp^2 / 4 |d2I/dlambda2_k| fitted
  by least squares over the interior centres (the magnitude only: the sign
  of this relation flips between optically thin and saturated lines);
* azimuth (our reading of Auer et al. 1977): from the linear polarisation
  of the line wings, where the sigma components fix its sign and the
  magneto-optical rotation is small: 2 psi = atan2(sum w_k U_k,
  sum w_k Q_k) with w_k = (c_k - cbar)^4, cbar the mean centre; with more
  than 8 samples (spectra reaching into the continuum, where the samples
  carry only noise) w_k is multiplied by the squared relative line depth
  ((I_c - I_k) / max_j (I_c - I_j))^2, which vanishes there;
* the sign s_V of the longitudinal relation is that of the synthesis
  convention (``SIGN_V``), pinned by the tests on weak-field profiles;
* B = sqrt(B_par^2 + B_perp^2), gamma = atan2(B_perp, B_par);
* polarisation level: max_k sqrt(Q_k^2 + U_k^2 + V_k^2) / I_c, I_c the
  largest Stokes I sample;
* for a stand-alone initial model (no network) the line-of-sight velocity
  is the centre of gravity of the line depth I_c - I_k over the filter
  centres (not in the paper, which takes v from the network), and the
  other parameters are the standard guess.
"""
from __future__ import annotations

import numpy as np

from . import lm, me

# Sign of the longitudinal weak-field relation in the synthesis convention
# of me.py (blue sigma component at -dlambda_B).
SIGN_V = -1.0
PAPER_POL_THRESHOLD = 0.06


def filter_centres(filters, x):
    T = np.asarray(filters, dtype=np.float64)
    return (T * np.asarray(x, dtype=np.float64)[None, :]).sum(1) / T.sum(1)


def _derivatives(I, c):
    """dI/dc at every centre and d2I/dc2 at the interior ones (c increasing)."""
    n = c.size
    d1 = np.empty_like(I)
    d1[:, 0] = (I[:, 1] - I[:, 0]) / (c[1] - c[0])
    d1[:, -1] = (I[:, -1] - I[:, -2]) / (c[-1] - c[-2])
    for k in range(1, n - 1):
        d1[:, k] = (I[:, k + 1] - I[:, k - 1]) / (c[k + 1] - c[k - 1])
    d2 = np.zeros_like(I)
    for k in range(1, n - 1):
        right = (I[:, k + 1] - I[:, k]) / (c[k + 1] - c[k])
        left = (I[:, k] - I[:, k - 1]) / (c[k] - c[k - 1])
        d2[:, k] = 2.0 * (right - left) / (c[k + 1] - c[k - 1])
    return d1, d2


def weak_field(obs, filters, x, line):
    """B, gamma, psi and the polarisation level of each pixel."""
    obs = np.asarray(obs, dtype=np.float64)
    nf = obs.shape[1] // 4
    c = filter_centres(filters, x)
    order = np.argsort(c, kind="stable")
    c = c[order]
    I, Q, U, V = (obs[:, s * nf:(s + 1) * nf][:, order] for s in range(4))
    C = me.zeeman_mA_per_G(line["lambda0_A"], line["geff"])
    d1, d2 = _derivatives(I, c)
    den1 = (d1 * d1).sum(1)
    bpar = np.where(den1 > 0, (V * d1).sum(1) / np.where(den1 > 0, den1, 1.0), 0.0) / (SIGN_V * C)
    inner = slice(1, nf - 1)
    den2 = (d2[:, inner] ** 2).sum(1)
    safe = np.where(den2 > 0, den2, 1.0)
    qa = np.where(den2 > 0, (Q[:, inner] * d2[:, inner]).sum(1) / safe, 0.0)
    ub = np.where(den2 > 0, (U[:, inner] * d2[:, inner]).sum(1) / safe, 0.0)
    bperp = 2.0 * np.sqrt(np.sqrt(qa * qa + ub * ub)) / C
    wk = np.broadcast_to((c - c.mean()) ** 4, I.shape)
    if nf > 8:
        depth = I.max(1, keepdims=True) - I
        dmax = depth.max(1, keepdims=True)
        rel = np.where(dmax > 0, depth / np.where(dmax > 0, dmax, 1.0), 0.0)
        wk = wk * rel * rel
    psi = np.mod(0.5 * np.degrees(np.arctan2((U * wk).sum(1), (Q * wk).sum(1))), 180.0)
    B = np.hypot(bpar, bperp)
    gamma = np.degrees(np.arctan2(bperp, bpar))
    ic = I.max(1)
    pol = np.sqrt(Q * Q + U * U + V * V).max(1) / ic
    return {"B": B, "gamma": gamma, "psi": psi, "pol": pol, "bpar": bpar, "bperp": bperp}


def cog_velocity(obs, filters, x, line):
    """Line-of-sight velocity [km/s] from the centre of gravity of I_c - I_k."""
    obs = np.asarray(obs, dtype=np.float64)
    nf = obs.shape[1] // 4
    c = filter_centres(filters, x)
    I = obs[:, :nf]
    depth = I.max(1)[:, None] - I
    tot = depth.sum(1)
    lam = np.where(tot > 0, (depth * c[None, :]).sum(1) / np.where(tot > 0, tot, 1.0), 0.0)
    return lam / me.doppler_mA_per_kms(line["lambda0_A"])


def initial_models(obs, filters, x, line):
    """Stand-alone initial models [npix, 10]: weak-field B, gamma, psi,
    centre-of-gravity v, the standard guess for the rest."""
    obs = np.asarray(obs, dtype=np.float64)
    nf = obs.shape[1] // 4
    mu = float(line.get("mu", 1.0))
    m = lm.standard_guess(obs, nf, mu)
    wf = weak_field(obs, filters, x, line)
    m[:, me.B] = wf["B"]
    m[:, me.GAMMA] = wf["gamma"]
    m[:, me.PSI] = wf["psi"]
    m[:, me.VLOS] = cog_velocity(obs, filters, x, line)
    return lm.apply_bounds(m)


def merge_paper(init_nn, obs, filters, x, line, threshold=PAPER_POL_THRESHOLD):
    """The paper's combination: the network's model, with B and gamma from
    the weak-field estimate where the polarisation is below ``threshold``
    and psi from the linear-polarisation estimate everywhere."""
    m = np.array(init_nn, dtype=np.float64, copy=True)
    wf = weak_field(obs, filters, x, line)
    low = wf["pol"] < threshold
    m[low, me.B] = wf["B"][low]
    m[low, me.GAMMA] = wf["gamma"][low]
    m[:, me.PSI] = wf["psi"]
    return lm.apply_bounds(m)
