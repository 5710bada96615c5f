"""Levenberg-Marquardt inversion of the Milne-Eddington model, FP64 (oracle).

TEST INFRASTRUCTURE ONLY -- see the package docstring.

The algorithm follows Sec. 2 (Eqs. 1-6), Sec. 4.2 (Table 2) and Sec. 4.4
(Fig. 6) step by step, for many independent pixels at once (numpy arrays
over pixels; each pixel keeps its own model, damping and iteration count,
exactly as if it were inverted alone).

Readings of points the paper leaves open or prints garbled:
* Eqs. 3-4 print H_ij as a product of chi-square gradients; read as the
  Gauss-Newton matrix A = J^T W J with diagonal A_ii (1 + eps), the form of
  the Levenberg-Marquardt recipe the paper cites (Press et al.).
* The step solves (A + eps diag(A)) delta = J^T W r; it is computed in the
  Jacobi-scaled form (A_s + eps I) y = D^-1/2 g, delta = D^-1/2 y, with
  D = diag(A), by SVD with singular values below 1e-12 * max zeroed (the
  paper's Svdcmp/Svbksb).  A free parameter whose Jacobian column is exactly
  zero (D_ii = 0) is held for that step.
* Table 2's overlapping rows: on success eps > 1e4 -> /100,
  1e-4 <= eps <= 1e4 -> /10, eps < 1e-4 -> /2; on failure eps < 1e-4 -> x100,
  1e-4 <= eps <= 1e4 -> x2, eps > 1e4 -> x10.  The paper gives no floor; eps
  is kept >= 1e-9, so the Jacobi-scaled damped matrix (unit diagonal) has
  every eigenvalue >= 1e-9 and the step never needs truncation; eps > 1e12
  ends the iteration (no decrease is possible).
* A trial is successful iff chi2_trial < chi2_best (strict); equality or a
  non-finite chi2 is a failure (Fig. 6: derivatives only after a success).
* Stopping (the paper runs a fixed count): a pixel is converged when a
  successful step lowers chi2 by less than ``conv_rtol`` relative while the
  step was close to Gauss-Newton (eps_used <= ``conv_eps``), or when eps
  exceeds 1e12 after a failure (no decrease possible, status STALLED);
  otherwise it stops at ``max_iter`` trial steps (status MAXITER).  The
  iteration count is the number of trial solves (the paper's Svdcmp count).
* Without given initial models the iteration starts from the filtergram
  models of ``oracle.init`` when ``wfa_pol`` > 0 (Sec. 5), else from the
  standard initial guess (the paper uses ANN/weak-field guesses):
  B = 500 G, gamma = 60 deg, psi = 45 deg, eta0 = 10, dlambdaD = 35 mA,
  a = 0.25, v = 0, S0 = 0.25 Ic, S1 = 0.75 Ic / mu, alpha = 1, where Ic is the
  largest observed Stokes I sample.
* Bounds after each step: B < 0 -> (-B, 180 - gamma); gamma reflected into
  [0, 180] (the profiles depend on sin^2 gamma and cos gamma only);
  psi mod 180; B <= 6000 G; eta0 in [0.01, 500]; dlambdaD in [5, 150] mA;
  a in [0, 5]; |v| <= 20 km/s; S0, S1 in [0, 2]; alpha in [0, 1].
* The filling factor alpha (Sec. 2) is held at 1 unless bit 9 of
  ``free_mask`` is set; free, it joins the solve with the column
  S_mag - S_mag(B=0) (the other columns mixed alpha : 1 - alpha).
* Covariance: (J^T W J)^+ at the final model (eps = 0), computed in the
  Jacobi-scaled form with the same SVD truncation, zero for held
  parameters.
* Hessian reuse near the minimum (Sec. 4.4, Fig. 6, optional): the paper
  skips the Hessian when "chi2 << 1", a level the Eq. 1 normalisation never
  reaches (chi2 ~ 1 at the fit).  Read here as: an accepted step is close to
  the minimum when it lowered chi2 by less than ``hess_reuse`` relative;
  when it and the previous accepted step both are, J^T W J is kept from the
  previous model and only J^T W r is rebuilt (the derivatives are still
  computed, Fig. 6).  The covariance then comes from the matrix in use.
  0 disables it.  A restart clears the "previous step close" state.
* Randomised restarts (Sec. 4.2, optional, ``restarts`` a bit mask): every
  pixel runs exactly ``max_iter`` iterations.  A restart is due (bit 0)
  when a step meets the convergence test or the pixel stalls, (bit 1, the
  paper's (a)) at iteration 10 of the inversion if chi2 is not below a
  tenth of its initial value, (bit 2, the paper's (b)) when 5 trials in a
  row have failed.  The paper states (a) for "the first 10 iterations", so
  it is tested once, with the best chi2 so far, not in every segment.  The restart replaces the next
  trial: the best model of all segments so far, perturbed with amplitudes
  proportional to the restart count k (uniform in B +- 150k G,
  gamma +- 10k deg, psi +- 15k deg, ln eta0 +- 0.25k, dlambdaD +- 4k mA,
  a +- 0.05k, v +- 0.25k km/s; S0, S1 and held parameters untouched; bounds
  applied), is evaluated and taken as the start of a new segment whatever
  its chi2 (a non-finite one is retried with k + 1), with the damping reset
  to eps0.  It counts as one iteration.  The result is the best model of
  all segments (with its covariance); the status is CONVERGED if any
  segment converged, else STALLED if any stalled, else MAXITER.  The
  uniforms are SplitMix64 outputs (Steele, Lea & Flood 2014) at counter
  (pixel << 24) | (k << 4) | p for parameter p, keyed by ``seed``; pixel is
  the pixel's index in the call.
"""
from __future__ import annotations

import numpy as np

from . import me

NPAR = 10
DEFAULT_FREE = 0x1FF  # B..S1 free, alpha held

CONVERGED, MAXITER, STALLED, BAD_INPUT, NAN_STATE = 0, 1, 2, 3, 4

EPS_MIN, EPS_MAX = 1e-9, 1e12
SVD_RCOND = 1e-12

STANDARD_GUESS = np.array([500.0, 60.0, 45.0, 10.0, 35.0, 0.25, 0.0, 0.25, 0.75, 1.0])


def chi2(obs, syn, w, nfree):
    """Eq. 1: sum_ij (I_obs - I_syn)^2 w_ij^2 / sigma_ij^2 / (4L - F); the
    combined factor w^2/sigma^2 is the ``w`` array."""
    n_obs = obs.shape[-1]
    r = obs - syn
    return (w * r * r).sum(-1) / (n_obs - nfree)


def eps_update(eps, success):
    """Table 2: new damping from the old one and the outcome of the step."""
    eps = np.asarray(eps, dtype=np.float64)
    dec = np.where(eps > 1e4, eps / 100.0, np.where(eps >= 1e-4, eps / 10.0, eps / 2.0))
    inc = np.where(eps < 1e-4, eps * 100.0, np.where(eps <= 1e4, eps * 2.0, eps * 10.0))
    return np.clip(np.where(success, dec, inc), EPS_MIN, None)


def standard_guess(obs, nfilt, mu=1.0):
    ic = obs[:, :nfilt].max(axis=1)
    m = np.tile(STANDARD_GUESS, (obs.shape[0], 1))
    m[:, me.S0] = 0.25 * ic
    m[:, me.S1] = 0.75 * ic / mu
    return m


def apply_bounds(m):
    m = m.copy()
    neg = m[:, me.B] < 0
    m[neg, me.B] = -m[neg, me.B]
    m[neg, me.GAMMA] = 180.0 - m[neg, me.GAMMA]
    g = np.mod(m[:, me.GAMMA], 360.0)
    m[:, me.GAMMA] = np.where(g > 180.0, 360.0 - g, g)
    m[:, me.PSI] = np.mod(m[:, me.PSI], 180.0)
    m[:, me.B] = np.minimum(m[:, me.B], 6000.0)
    m[:, me.ETA0] = np.clip(m[:, me.ETA0], 0.01, 500.0)
    m[:, me.DLD] = np.clip(m[:, me.DLD], 5.0, 150.0)
    m[:, me.DAMP] = np.clip(m[:, me.DAMP], 0.0, 5.0)
    m[:, me.VLOS] = np.clip(m[:, me.VLOS], -20.0, 20.0)
    m[:, me.S0] = np.clip(m[:, me.S0], 0.0, 2.0)
    m[:, me.S1] = np.clip(m[:, me.S1], 0.0, 2.0)
    m[:, me.ALPHA] = np.clip(m[:, me.ALPHA], 0.0, 1.0)
    return m


def normal_equations(J, r, w, free):
    """A = J^T W J and g = J^T W r over the free parameters (Eqs. 2-4 read as
    Gauss-Newton); held parameters get zero rows and columns."""
    Jf = J * free[None, None, :]
    A = np.einsum("poi,po,poj->pij", Jf, w, Jf)
    g = np.einsum("poi,po,po->pi", Jf, w, r)
    return A, g


def _scaled(A, free):
    d = np.diagonal(A, axis1=1, axis2=2)
    held = (~free[None, :]) | ~(d > 0) | ~np.isfinite(d)
    s = np.where(held, 0.0, 1.0 / np.sqrt(np.where(held, 1.0, d)))
    As = A * s[:, :, None] * s[:, None, :]
    return As, s, held


def _svd_solve(Mx, b):
    U, S, Vt = np.linalg.svd(Mx)
    keep = S > SVD_RCOND * S[:, :1]
    Sinv = np.where(keep, 1.0 / np.where(keep, S, 1.0), 0.0)
    return np.einsum("pji,pj->pi", Vt, Sinv * np.einsum("pji,pj->pi", U, b))


def damped_step(A, g, eps, free):
    """Eqs. 4-5: delta solving (A + eps diag A) delta = g (Jacobi-scaled, SVD)."""
    As, s, held = _scaled(A, free)
    n = A.shape[-1]
    Mx = As + eps[:, None, None] * np.eye(n)[None]
    Mx[held] = 0.0                       # rows of held parameters
    Mx = np.where(held[:, None, :], 0.0, Mx)
    Mx = Mx + np.eye(n)[None] * held[:, :, None]
    y = _svd_solve(Mx, np.where(held, 0.0, g * s))
    return np.where(held, 0.0, s * y)


def covariance(A, free):
    """(J^T W J)^+ in parameter units, held parameters zero."""
    As, s, held = _scaled(A, free)
    n = A.shape[-1]
    Mx = np.where(held[:, None, :] | held[:, :, None], 0.0, As)
    U, S, Vt = np.linalg.svd(Mx)
    keep = S > SVD_RCOND * S[:, :1]
    Sinv = np.where(keep, 1.0 / np.where(keep, S, 1.0), 0.0)
    P = np.einsum("pki,pk,pkj->pij", Vt, Sinv, Vt)
    return P * s[:, :, None] * s[:, None, :]


# --- Sec. 4.2: randomised restarts ------------------------------------------

_M64 = (1 << 64) - 1
SPLITMIX_GAMMA = 0x9E3779B97F4A7C15
RESTART_AMPLITUDE = np.array([150.0, 10.0, 15.0, 0.25, 4.0, 0.05, 0.25])  # per unit k; eta0 in ln
RESTART_AT_CONVERGENCE, RESTART_A, RESTART_B = 1, 2, 4
RESTART_A_ITER, RESTART_A_FACTOR, RESTART_B_FAILS = 10, 10.0, 5


def splitmix64(seed, counter):
    """The counter-th output (0-based) of SplitMix64 started from ``seed``:
    the state advanced counter+1 times by the golden-ratio increment, then
    the variant-13 64-bit finaliser (xor-shift 30, 27, 31 with the two odd
    multipliers).  Python integers, so the wrap-around is explicit."""
    z = (int(seed) + (int(counter) + 1) * SPLITMIX_GAMMA) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def restart_uniform(seed, pix, k, p):
    """Uniform in [0, 1) from the top 53 bits of one SplitMix64 output."""
    return (splitmix64(seed, (int(pix) << 24) | (int(k) << 4) | int(p)) >> 11) * 2.0 ** -53


def restart_model(m, pix, k, seed, free):
    """Perturbed copy of models m [n, 10] for restart number k of pixels pix."""
    out = np.array(m, dtype=np.float64, copy=True)
    for i, (px, kk) in enumerate(zip(np.atleast_1d(pix), np.broadcast_to(k, len(out)))):
        for p in range(7):
            if not free[p]:
                continue
            r = 2.0 * restart_uniform(seed, px, kk, p) - 1.0
            amp = RESTART_AMPLITUDE[p] * kk * r
            if p == me.ETA0:
                out[i, p] *= np.exp(amp)
            else:
                out[i, p] += amp
    return apply_bounds(out)


def invert(obs, w, filters, x, line, init=None, max_iter=50, conv_rtol=1e-4,
           conv_eps=1.0, eps0=1.0, free_mask=DEFAULT_FREE, restarts=0, seed=0,
           hess_reuse=0.0, wfa_pol=0.0, trace=False):
    """Invert observed Stokes [npix, 4*nfilt] with weights w^2/sigma^2.

    Returns a dict with params [npix,10], chi2 [npix], iters [npix],
    status [npix], cov [npix,10,10], accepted [npix] (and, with restarts,
    restarts [npix]).
    """
    obs = np.asarray(obs, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    npix, n_obs = obs.shape
    nfilt = n_obs // 4
    mu = float(line.get("mu", 1.0))
    free = np.array([(free_mask >> k) & 1 for k in range(NPAR)], dtype=bool)
    nfree = int(free.sum())

    bad = ~np.isfinite(obs).all(1) | ~np.isfinite(w).all(1) | ~(w.sum(1) > 0)
    if init is None and wfa_pol > 0:
        from . import init as init_mod   # Sec. 5: models from the filtergrams
        m = init_mod.initial_models(np.where(np.isfinite(obs), obs, 0.0), filters, x, line)
    elif init is None:
        m = standard_guess(np.where(np.isfinite(obs), obs, 0.0), nfilt, mu)
    else:
        m = np.asarray(init, dtype=np.float64).copy()
        bad |= ~np.isfinite(m).all(1)
        m = np.where(np.isfinite(m), m, STANDARD_GUESS[None, :])
    if not free[me.ALPHA]:
        m[:, me.ALPHA] = 1.0          # the filling factor held at 1
    m = apply_bounds(m)
    obs_s = np.where(bad[:, None], 0.0, obs)
    w_s = np.where(bad[:, None], 0.0, w)

    def model(mm, jac):
        out = me.synth(mm, filters, x, line, jacobian=jac, alpha_jacobian=bool(free[me.ALPHA]))
        if jac:
            s, J = out
            return s.reshape(len(mm), -1), J.reshape(len(mm), n_obs, NPAR)
        return out.reshape(len(mm), -1)

    syn, J = model(m, True)
    c2 = chi2(obs_s, syn, w_s, nfree)
    A, g = normal_equations(J, obs_s - syn, w_s, free)
    eps = np.full(npix, float(eps0))
    iters = np.zeros(npix, dtype=np.int64)
    nacc = np.zeros(npix, dtype=np.int64)
    status = np.full(npix, MAXITER, dtype=np.int64)
    status[bad] = BAD_INPUT
    nan0 = ~bad & ~np.isfinite(c2)
    status[nan0] = NAN_STATE
    done = bad | nan0
    hist = []
    near_prev = np.zeros(npix, dtype=bool)   # previous accepted step close to the minimum
    if restarts:
        best_m, best_c2, best_A, best_g = m.copy(), c2.copy(), A.copy(), g.copy()
        c2_first = c2.copy()
        nfail = np.zeros(npix, dtype=np.int64)
        nrestart = np.zeros(npix, dtype=np.int64)
        ever_conv = np.zeros(npix, dtype=bool)
        ever_stall = np.zeros(npix, dtype=bool)
        pending = np.zeros(npix, dtype=bool)

    for _ in range(max_iter):
        act = np.flatnonzero(~done)
        if act.size == 0:
            break
        rs = np.zeros(0, dtype=np.int64)
        if restarts:
            rs = act[pending[act]]
            act = act[~pending[act]]
            if rs.size:
                # the restart pass: perturbed best model, a new segment
                nrestart[rs] += 1
                mt = restart_model(best_m[rs], rs, nrestart[rs], seed, free)
                sr, Jr = model(mt, True)
                cr = chi2(obs_s[rs], sr, w_s[rs], nfree)
                iters[rs] += 1
                fin = np.isfinite(cr)
                ok_r = rs[fin]
                m[ok_r], c2[ok_r] = mt[fin], cr[fin]
                Ar, gr = normal_equations(Jr[fin], obs_s[ok_r] - sr[fin], w_s[ok_r], free)
                A[ok_r], g[ok_r] = Ar, gr
                nfail[ok_r] = 0
                near_prev[ok_r] = False
                eps[ok_r] = float(eps0)
                pending[ok_r] = False        # a non-finite restart is retried with k + 1
        delta = damped_step(A[act], g[act], eps[act], free)
        mt = apply_bounds(m[act] + delta)
        st = model(mt, False)
        ct = chi2(obs_s[act], st, w_s[act], nfree)
        iters[act] += 1
        ok = np.isfinite(ct) & (ct < c2[act])
        eps_used = eps[act].copy()
        eps[act] = eps_update(eps_used, ok)
        acc = act[ok]
        conv_now = np.zeros(0, dtype=np.int64)
        if acc.size:
            rel = (c2[acc] - ct[ok]) / c2[acc]
            m[acc] = mt[ok]
            c2[acc] = ct[ok]
            nacc[acc] += 1
            sa, Ja = model(m[acc], True)
            Aa, ga = normal_equations(Ja, obs_s[acc] - sa, w_s[acc], free)
            near = rel < hess_reuse
            keep = near & near_prev[acc]          # reuse J^T W J of the previous model
            A[acc[~keep]] = Aa[~keep]
            g[acc] = ga
            near_prev[acc] = near
            conv = (rel < conv_rtol) & (eps_used[ok] <= conv_eps)
            conv_now = acc[conv]
        rej = act[~ok]
        stall_now = rej[eps[rej] >= EPS_MAX]
        if restarts:
            moved = np.concatenate([acc, rs])
            nb = moved[c2[moved] < best_c2[moved]]
            best_m[nb], best_c2[nb], best_A[nb], best_g[nb] = m[nb], c2[nb], A[nb], g[nb]
            nfail[acc] = 0
            nfail[rej] += 1
            ever_conv[conv_now] = True
            ever_stall[stall_now] = True
            trig = np.zeros(npix, dtype=bool)
            if restarts & RESTART_AT_CONVERGENCE:
                trig[conv_now] = True
                trig[stall_now] = True
            else:                                # a converged or stalled pixel stops
                status[conv_now] = CONVERGED
                status[stall_now] = STALLED
                done[conv_now] = True
                done[stall_now] = True
            if restarts & RESTART_A:
                trig[act] |= (iters[act] == RESTART_A_ITER) & ~(best_c2[act] <= c2_first[act] / RESTART_A_FACTOR)
            if restarts & RESTART_B:
                trig[act] |= nfail[act] >= RESTART_B_FAILS
            pending |= trig & ~done
            done |= iters >= max_iter
        else:
            status[conv_now] = CONVERGED
            done[conv_now] = True
            status[stall_now] = STALLED
            done[stall_now] = True
        if trace:
            hist.append((act.size + rs.size, acc.size))

    out = {"accepted": nacc, "iters": iters}
    if restarts:
        ran = ~bad & ~nan0
        m = np.where(ran[:, None], best_m, m)
        c2 = np.where(ran, best_c2, c2)
        A = np.where(ran[:, None, None], best_A, A)
        status[ran] = np.where(ever_conv[ran], CONVERGED,
                               np.where(ever_stall[ran], STALLED, MAXITER))
        out["restarts"] = nrestart
    cov = covariance(A, free)
    out.update({"params": m, "chi2": c2, "status": status, "cov": cov})
    if trace:
        out["trace"] = hist
    return out


def invert_mixed(obs, w, filters, x, line, blob, nn_cap=20, plain_cap=50, chi2_flag=3.0,
                 flag_unconverged=True, conf_route=np.inf, operand_round=None, wfa_pol=0.0,
                 plain_wfa_pol=0.0, **kw):
    """Network-initialised inversion with plain re-inversion of flagged pixels.

    The network (FP64 forward of ``blob``; with ``operand_round`` every
    layer's operands rounded first, the tensor-core reading) gives the
    initial models and the confidence output (column 10 of its outputs, its
    estimate of the log mean squared error of the standardised guess).
    Pixels whose confidence output is above ``conf_route`` (or not a number)
    are routed: they skip the LM run from the guess and are inverted from the
    standard guess only.  The others run LM with ``nn_cap``; those ending
    with chi2 > chi2_flag (or, with flag_unconverged, not converged; STALLED
    counts as converged) are inverted again from the standard guess with
    ``plain_cap`` and keep the lower chi2; iteration counts add.  A routed
    pixel keeps the plain result; if that has no finite chi2 it ends in
    NAN_STATE with the network's guess and a zero covariance.
    With ``wfa_pol`` > 0 the network's guess is combined the paper's way
    (Sec. 5): weak-field B and gamma below that polarisation level, the
    wing azimuth everywhere (``oracle.init.merge_paper``); with
    ``plain_wfa_pol`` > 0 the re-inversion starts from the filtergram models
    (``oracle.init.initial_models``) instead of the standard guess."""
    from . import init as init_mod, mlp
    mu = float(line.get("mu", 1.0))
    npix = obs.shape[0]
    weights, stats = mlp.unpack(blob)
    y, _ = mlp.forward(weights, mlp.features(obs, stats), operand_round=operand_round)
    init = mlp.decode(y, obs, stats, mu)
    conf = y[:, mlp.NOUT_PARAM]
    if wfa_pol > 0:
        init = init_mod.merge_paper(init, obs, filters, x, line, wfa_pol)
    routed = ~(conf <= conf_route)
    run = np.flatnonzero(~routed)
    out = {"params": init.copy(), "chi2": np.full(npix, np.inf),
           "iters": np.zeros(npix, dtype=np.int64), "accepted": np.zeros(npix, dtype=np.int64),
           "status": np.full(npix, NAN_STATE, dtype=np.int64), "cov": np.zeros((npix, NPAR, NPAR))}
    if run.size:
        r = invert(obs[run], w[run], filters, x, line, init=init[run], max_iter=nn_cap, **kw)
        for k in ("params", "chi2", "iters", "accepted", "status", "cov"):
            out[k][run] = r[k]
    st = out["status"]
    conv = np.isin(st, (CONVERGED, STALLED))
    flag = routed | ((st != BAD_INPUT) &
                     ((flag_unconverged & ~conv) | ~(out["chi2"] <= chi2_flag)))
    out["flagged"] = flag.astype(np.int32)
    out["routed"] = routed.astype(np.int32)
    out["confidence"] = conf
    if flag.any():
        ids = np.flatnonzero(flag)
        q = invert(obs[ids], w[ids], filters, x, line, init=None, max_iter=plain_cap,
                   wfa_pol=plain_wfa_pol, **kw)
        out["iters"][ids] += q["iters"]
        out["accepted"][ids] += q["accepted"]
        plain_ok = (q["status"] != NAN_STATE) & np.isfinite(q["chi2"])
        nn_ok = (st[ids] != NAN_STATE) & np.isfinite(out["chi2"][ids])
        take = plain_ok & (~nn_ok | (q["chi2"] < out["chi2"][ids]))
        for k in ("params", "chi2", "status", "cov"):
            out[k][ids[take]] = q[k][take]
    return out


# --- Sec. 4.3: weights for full-disk maps ----------------------------------

ICONT_MU_COEFFS = (0.33644, 1.30590, -1.79238, 2.45050, -1.89979, 0.59943)


def icont_mu(mu):
    """Eq. 15: continuum intensity versus mu near 6173 A (disk centre = 1)."""
    mu = np.asarray(mu, dtype=np.float64)
    return sum(c * mu ** k for k, c in enumerate(ICONT_MU_COEFFS))


def limb_weights(obs, mu, ic0, sigma, nfilt=6):
    """Eq. 14 weights as w^2 / sigma^2 per observable [npix, 4*nfilt]:
    w_I = 0.7778 |I_cont(mu) - I_cont(x,y)| + 0.3, w_Q = w_U = w_V = 1, with
    I_cont(x,y) the pixel's largest Stokes I sample divided by the disk-centre
    continuum ic0; sigma[4] is the noise of I, Q, U, V."""
    obs = np.asarray(obs, dtype=np.float64)
    ic = obs[:, :nfilt].max(axis=1) / ic0
    wI = 0.7778 * np.abs(icont_mu(mu) - ic) + 0.3
    w = np.ones((obs.shape[0], 4))
    w[:, 0] = wI
    s = np.asarray(sigma, dtype=np.float64)[None, :]
    return np.repeat(w * w / (s * s), nfilt, axis=1)
