"""Per-parameter error of a GPU inversion against the FP64 oracle's, the
report the parity tests print and the benchmark's oracle leg attaches to its
line.  Comparison only (no method arithmetic)."""
from __future__ import annotations

import numpy as np

NAMES = ("B", "gamma", "psi", "eta0", "dlambdaD", "a", "vlos", "S0", "S1")
# the stated tolerances: |dB| <= 1 G, |dgamma|, |dpsi| <= 0.05 deg, chi2 <= 1e-3 relative
TOL = {"B": 1.0, "gamma": 0.05, "psi": 0.05, "chi2_rel": 1e-3}
CONVERGED = 0


def param_delta(a, b):
    """|a - b| per parameter [n, 9]; psi compared modulo 180 degrees."""
    d = np.abs(np.asarray(a, dtype=np.float64)[:, :9] - np.asarray(b, dtype=np.float64)[:, :9])
    d[:, 2] = np.abs(np.mod(d[:, 2] + 90.0, 180.0) - 90.0)
    return d


def _stats(v):
    if v.size == 0:
        return {"n": 0}
    return {"n": int(v.size), "max": float(v.max()), "p99": float(np.percentile(v, 99)),
            "median": float(np.median(v))}


def error_table(gpu: dict, ref: dict, well_determined=None) -> dict:
    """Errors over the pixels CONVERGED in both runs: max / p99 / median of
    |delta| for every parameter and for chi2 (relative), the fraction within
    the stated tolerances, and the split of the chi2 mismatches into equal and
    different iteration counts (a different count marks trajectories that
    parted: an FP32 vs FP64 near-tie)."""
    sg, sr = np.asarray(gpu["status"]), np.asarray(ref["status"])
    both = (sg == CONVERGED) & (sr == CONVERGED)
    d = param_delta(gpu["params"], ref["params"])[both]
    cg = np.asarray(gpu["chi2"], dtype=np.float64)[both]
    cr = np.asarray(ref["chi2"], dtype=np.float64)[both]
    rel = np.abs(cg / cr - 1.0)
    same_it = (np.asarray(gpu["iters"]) == np.asarray(ref["iters"]))[both]
    out = {"pixels": int(sg.size), "converged_both": int(both.sum()),
           "converged_gpu": float((sg == CONVERGED).mean()),
           "converged_oracle": float((sr == CONVERGED).mean()),
           "chi2_rel": _stats(rel),
           "chi2_within_tol": float((rel <= TOL["chi2_rel"]).mean()) if rel.size else None,
           "chi2_mismatch_equal_iters": int(((rel > TOL["chi2_rel"]) & same_it).sum()),
           "chi2_mismatch_other_iters": int(((rel > TOL["chi2_rel"]) & ~same_it).sum()),
           "params": {}}
    for j, nm in enumerate(NAMES):
        e = _stats(d[:, j])
        if nm in TOL:
            e["within_tol"] = float((d[:, j] <= TOL[nm]).mean()) if d.shape[0] else None
        out["params"][nm] = e
    if well_determined is not None:
        wd = np.asarray(well_determined)[both]
        ok = ((d[:, 0] <= TOL["B"]) & (d[:, 1] <= TOL["gamma"]) & (d[:, 2] <= TOL["psi"]))
        out["well_determined"] = int(wd.sum())
        out["field_within_tol_well_determined"] = float(ok[wd].mean()) if wd.any() else None
    return out


def well_determined(ref: dict) -> np.ndarray:
    """Pixels whose field the oracle pins down: B >= 100 G and the oracle's
    standard errors of gamma and psi below 5 degrees."""
    cov = np.asarray(ref["cov"], dtype=np.float64)
    sg = np.sqrt(np.maximum(cov[:, 1, 1], 0.0))
    sp = np.sqrt(np.maximum(cov[:, 2, 2], 0.0))
    return (np.asarray(ref["params"])[:, 0] >= 100.0) & (sg < 5.0) & (sp < 5.0)


def format_table(t: dict) -> str:
    rows = [f"pixels {t['pixels']}, converged in both {t['converged_both']} "
            f"(gpu {t['converged_gpu']:.3f}, oracle {t['converged_oracle']:.3f})"]
    c = t["chi2_rel"]
    if c.get("n"):
        rows.append(f"chi2 rel: max {c['max']:.2e} p99 {c['p99']:.2e} median {c['median']:.2e} "
                    f"within 1e-3 {t['chi2_within_tol']:.4f} (mismatches: equal iterations "
                    f"{t['chi2_mismatch_equal_iters']}, other {t['chi2_mismatch_other_iters']})")
    for nm, e in t["params"].items():
        if e.get("n"):
            w = f" within {e['within_tol']:.4f}" if "within_tol" in e else ""
            rows.append(f"{nm:9s} max {e['max']:.3e} p99 {e['p99']:.3e} median {e['median']:.3e}{w}")
    if "well_determined" in t:
        rows.append(f"well determined {t['well_determined']}: field within tolerance "
                    f"{t['field_within_tol_well_determined']}")
    return "\n".join(rows)
