"""Milne-Eddington synthesis with analytic derivatives, FP64 (oracle).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

Parameter vector (per pixel, C-ABI order):
  0 B [G], 1 gamma [deg], 2 psi [deg], 3 eta0, 4 dlambdaD [mA], 5 a,
  6 vlos [km/s, positive = redshift], 7 S0, 8 S1, 9 alpha (filling factor).
These are the Milne-Eddington parameters of Sec. 2 with V_mac dropped.

Wavelengths are offsets x = lambda - lambda0 in mA.
"""
from __future__ import annotations

import numpy as np
from scipy.special import wofz

C_KMS = 299792.458
SQRT_PI = np.sqrt(np.pi)
DEG = np.pi / 180.0

# Parameter indices.
B, GAMMA, PSI, ETA0, DLD, DAMP, VLOS, S0, S1, ALPHA = range(10)


def zeeman_mA_per_G(lambda0_A: float, geff: float) -> float:
    """Sigma-component shift per gauss, Eq. 7: 4.66685e-10 * g_eff * lambda0^2 [mA/G]."""
    return 4.66685e-10 * geff * lambda0_A * lambda0_A


def doppler_mA_per_kms(lambda0_A: float) -> float:
    """Line-of-sight Doppler shift per km/s: lambda0 * v / c, in mA."""
    return lambda0_A * 1.0e3 / C_KMS


def voigt_faraday(a, u):
    """H(a,u) + i F(a,u) = w(u + i a), the Faddeeva function (Sec. 3.2).

    H is the Voigt function and F the Faraday-Voigt function, with the
    normalisation for which Eqs. 8-9 hold.  w comes from the library.
    """
    w = wofz(np.asarray(u, dtype=np.float64) + 1j * np.asarray(a, dtype=np.float64))
    return w.real, w.imag


def voigt_faraday_derivs(a, u, H, F):
    """Eqs. 8-9: alpha = dH/da = -dF/du, beta = dH/du = dF/da."""
    alpha = -2.0 / SQRT_PI + 2.0 * a * H + 2.0 * u * F
    beta = 2.0 * a * F - 2.0 * u * H
    return alpha, beta


def _profiles(p, x, line):
    """Normalised frequencies and Voigt/Faraday values of the pi, blue sigma
    and red sigma components, with their derivatives with respect to the
    parameters they depend on.  Shapes broadcast as [npix, nlam]."""
    cB = zeeman_mA_per_G(line["lambda0_A"], line["geff"])
    cv = doppler_mA_per_kms(line["lambda0_A"])
    Bf, dld, a, v = (p[:, k][:, None] for k in (B, DLD, DAMP, VLOS))
    x = np.asarray(x, dtype=np.float64)[None, :]
    u_pi = (x - cv * v) / dld
    u_zb = cB * Bf / dld
    comps = {}
    # blue sigma sits at -dlambda_B, red at +dlambda_B (Eq. 7 and text).
    for name, sign in (("p", 0.0), ("b", 1.0), ("r", -1.0)):
        u = u_pi + sign * u_zb
        H, F = voigt_faraday(a, u)
        al, be = voigt_faraday_derivs(a, u, H, F)
        # chain rule: d(H,F)/dq = (dH/du, dF/du) du/dq, with dH/du = beta,
        # dF/du = -alpha, dH/da = alpha, dF/da = beta.
        du = {
            B: np.broadcast_to(sign * cB / dld, u.shape),
            DLD: -u / dld,
            VLOS: np.broadcast_to(-cv / dld, u.shape),
        }
        dH = {q: be * d for q, d in du.items()}
        dF = {q: -al * d for q, d in du.items()}
        dH[DAMP] = al
        dF[DAMP] = be
        comps[name] = (H, F, dH, dF)
    return comps


def _elements(p, comps):
    """Absorption-matrix elements (eta_I, eta_Q, eta_U, eta_V, rho_Q, rho_U,
    rho_V) of a normal Zeeman triplet and their derivatives with respect to
    every model parameter that enters them.

    eta_I = 1 + eta0/2 [phi_p sin^2g + (phi_b+phi_r)/2 (1+cos^2g)]
    eta_Q = eta0/2 [phi_p - (phi_b+phi_r)/2] sin^2g cos2psi
    eta_U = eta0/2 [phi_p - (phi_b+phi_r)/2] sin^2g sin2psi
    eta_V = eta0/2 [phi_r - phi_b] cos g
    and the rho's with the Faraday-Voigt function in place of phi.
    """
    eta0 = p[:, ETA0][:, None]
    g = p[:, GAMMA][:, None] * DEG
    ps = p[:, PSI][:, None] * DEG
    sg, cg = np.sin(g), np.cos(g)
    c2, s2 = np.cos(2 * ps), np.sin(2 * ps)

    def build(fp, fb, fr):
        lin = fp - 0.5 * (fb + fr)
        e_I = 0.5 * eta0 * (fp * sg ** 2 + 0.5 * (fb + fr) * (1 + cg ** 2))
        e_Q = 0.5 * eta0 * lin * sg ** 2 * c2
        e_U = 0.5 * eta0 * lin * sg ** 2 * s2
        e_V = 0.5 * eta0 * (fr - fb) * cg
        return e_I, e_Q, e_U, e_V

    Hp, Fp, dHp, dFp = comps["p"]
    Hb, Fb, dHb, dFb = comps["b"]
    Hr, Fr, dHr, dFr = comps["r"]
    eI, eQ, eU, eV = build(Hp, Hb, Hr)
    _, rQ, rU, rV = build(Fp, Fb, Fr)
    el = np.stack([1.0 + eI, eQ, eU, eV, rQ, rU, rV])  # [7, npix, nlam]

    d = {}
    # profile-shape parameters: differentiate phi/psi, keep geometry fixed.
    for q in (B, DLD, DAMP, VLOS):
        zero = np.zeros_like(Hp)
        dI, dQ, dU, dV = build(dHp.get(q, zero), dHb.get(q, zero), dHr.get(q, zero))
        _, dQr, dUr, dVr = build(dFp.get(q, zero), dFb.get(q, zero), dFr.get(q, zero))
        d[q] = np.stack([dI, dQ, dU, dV, dQr, dUr, dVr])
    # eta0 enters linearly.
    d[ETA0] = np.stack([eI, eQ, eU, eV, rQ, rU, rV]) / eta0
    # inclination (per degree).
    dsg2 = 2 * sg * cg * DEG          # d sin^2 g / d gamma_deg
    dcg = -sg * DEG                    # d cos g / d gamma_deg

    def build_g(fp, fb, fr):
        lin = fp - 0.5 * (fb + fr)
        e_I = 0.5 * eta0 * (fp * dsg2 + 0.5 * (fb + fr) * (-dsg2))
        e_Q = 0.5 * eta0 * lin * dsg2 * c2
        e_U = 0.5 * eta0 * lin * dsg2 * s2
        e_V = 0.5 * eta0 * (fr - fb) * dcg
        return e_I, e_Q, e_U, e_V

    gI, gQ, gU, gV = build_g(Hp, Hb, Hr)
    _, gQr, gUr, gVr = build_g(Fp, Fb, Fr)
    d[GAMMA] = np.stack([gI, gQ, gU, gV, gQr, gUr, gVr])
    # azimuth (per degree): only the Q/U elements rotate.
    z = np.zeros_like(Hp)
    d[PSI] = np.stack([z, -2 * DEG * eU, 2 * DEG * eQ, z, -2 * DEG * rU, 2 * DEG * rQ, z])
    return el, d


def propagation_matrix(el):
    """4x4 absorption (propagation) matrix from its seven elements [7, ...]."""
    eI, eQ, eU, eV, rQ, rU, rV = el
    K = np.empty(eI.shape + (4, 4))
    K[..., 0, :] = np.stack([eI, eQ, eU, eV], -1)
    K[..., 1, :] = np.stack([eQ, eI, rV, -rU], -1)
    K[..., 2, :] = np.stack([eU, -rV, eI, rQ], -1)
    K[..., 3, :] = np.stack([eV, rU, -rQ, eI], -1)
    return K


def _magnetic_unit(p, x, line, with_derivs):
    """y = K^{-1} e0 per (pixel, wavelength): the Stokes vector of the
    Milne-Eddington solution I = S0 e0 + mu S1 K^{-1} e0 divided by mu S1,
    without the S0 term.  With derivatives, dy/dq = -K^{-1} (dK/dq) y.
    Returns y [npix, nlam, 4] and {q: dy/dq}."""
    comps = _profiles(p, x, line)
    el, d = _elements(p, comps)
    K = propagation_matrix(el)
    e0 = np.zeros(K.shape[:-1])
    e0[..., 0] = 1.0
    y = np.linalg.solve(K, e0[..., None])[..., 0]
    dy = {}
    if with_derivs:
        for q, de in d.items():
            dK = propagation_matrix(de)
            rhs = -np.einsum("...ij,...j->...i", dK, y)
            dy[q] = np.linalg.solve(K, rhs[..., None])[..., 0]
    return y, dy


def synth(params, filters, x, line, jacobian: bool = False, alpha_jacobian: bool = False):
    """Filtered Stokes vector [npix, 4, nfilt] (and Jacobian [npix, 4, nfilt, 10]).

    S(x) = alpha * S_mag(x) + (1 - alpha) * S_mag(x; B=0) with
    S_mag = S0 e0 + mu S1 K^{-1} e0, then the filter convolution
    S_jk = sum_i T_k(x_i) S_j(x_i) (the instrument's 6 tuning positions).
    The B = 0 profile is computed when some alpha differs from 1, or with
    ``alpha_jacobian`` (the alpha column, S_mag - S_mag(B=0), needs it at
    alpha = 1 too); otherwise the alpha column is not meaningful.
    """
    p = np.atleast_2d(np.asarray(params, dtype=np.float64))
    T = np.asarray(filters, dtype=np.float64)
    mu = float(line.get("mu", 1.0))
    al = p[:, ALPHA]
    y, dy = _magnetic_unit(p, x, line, jacobian)
    needs_nm = np.any(al != 1.0) or (jacobian and alpha_jacobian)
    if needs_nm:
        pn = p.copy()
        pn[:, B] = 0.0
        yn, dyn = _magnetic_unit(pn, x, line, jacobian)
    else:
        yn, dyn = np.zeros_like(y), {q: np.zeros_like(y) for q in dy}
    a3 = al[:, None, None]
    ymix = a3 * y + (1 - a3) * yn                     # [npix, nlam, 4]
    tsum = T.sum(axis=1)                              # [nfilt]
    filt = lambda s: np.einsum("pls,kl->psk", s, T)  # noqa: E731
    s0 = p[:, S0][:, None, None]
    s1 = p[:, S1][:, None, None]
    e0k = np.zeros((1, 4, T.shape[0]))
    e0k[0, 0, :] = tsum
    line_part = filt(ymix)
    stokes = s0 * e0k + mu * s1 * line_part
    if not jacobian:
        return stokes
    J = np.zeros(stokes.shape + (10,))
    for q in (ETA0, DLD, DAMP, VLOS):
        J[..., q] = mu * s1 * filt(a3 * dy[q] + (1 - a3) * dyn[q])
    for q in (B, GAMMA, PSI):
        J[..., q] = mu * s1 * filt(a3 * dy[q])
    J[..., S0] = np.broadcast_to(e0k, stokes.shape)
    J[..., S1] = mu * line_part
    J[..., ALPHA] = mu * s1 * filt(y - yn)
    return stokes, J


def unfiltered(params, x, line):
    """Stokes vector on the wavelength grid, [npix, nlam, 4] (no filters)."""
    p = np.atleast_2d(np.asarray(params, dtype=np.float64))
    mu = float(line.get("mu", 1.0))
    y, _ = _magnetic_unit(p, x, line, False)
    if np.any(p[:, ALPHA] != 1.0):
        pn = p.copy()
        pn[:, B] = 0.0
        yn, _ = _magnetic_unit(pn, x, line, False)
        a3 = p[:, ALPHA][:, None, None]
        y = a3 * y + (1 - a3) * yn
    out = mu * p[:, S1][:, None, None] * y
    out[..., 0] += p[:, S0][:, None]
    return out
