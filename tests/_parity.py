"""Comparison of the CUDA path with the CPU FP64 oracle (shared by the GPU parity tests).

Tolerances (the targets of the mixed-precision and plain FP64 paths):
  mixed   SDF |err| <= 1e-4 m; gradient angle <= 0.1 deg; var_sdf relative <= 1e-3;
          var_f |err| <= 1e-3 * max(var_f, 1e-3) (var_f is cancellation-bound near the surface).
  fp64    relative <= 1e-9 with floor scale max(|ref|, 1e-3) for sdf, var_f; gradient components
          absolute <= 1e-9 (unit vector); var_sdf relative <= 1e-9.
Winner choice: where the GPU's winner differs from the oracle's, the query must carry the near-tie flag
(bit 2) on the GPU or in the oracle -- the mixed path sets it when another candidate's u lies within the
error bounds of the two FP32 evaluations -- and the GPU's winner must be an oracle candidate whose u is
within the SDF tolerance of the oracle's minimum; gradient and variances are then compared with the
oracle evaluated on the GPU's winner.
Exclusions (each counted): for the gradient angle only, medial-axis queries -- cancellation ratio
|sum_i a_i k'_i (x - x_i)| / sum_i |a_i| k'_i |x - x_i| < 1e-2 on the winner (the direction of a nearly
cancelling sum is ill-conditioned) -- and zero-gradient flags.
"""
import numpy as np

SDF_TOL = 1e-4
ANGLE_TOL_DEG = 0.1
VAR_SDF_REL = 1e-3
VAR_F_REL, VAR_F_FLOOR = 1e-3, 1e-3
F64_REL = 1e-9
MEDIAL_RATIO = 1e-2
# the FP32 adjoint: relative error of each query's d xq vector, and of the sample gradient d x (max over
# samples of the error, over the largest entry).  For a cotangent on sdf alone d xq is d sdf times the SDF's
# gradient: its direction is the forward gradient's (held to 0.1 deg = 1.75e-3 rad) and its magnitude
# |grad f'| / (lambda u f') carries the same FP32 conditioning (the cancellation in the sums over the winner's
# samples); the bound takes the direction tolerance for each of the two parts: 2 tan(0.1 deg) = 3.5e-3.
ADJ_REL = 3.5e-3


def cancellation_ratio(model, xq, cells):
    """Oracle-side conditioning of the gradient sum sum_i alpha_i w_i (x - x_i) for each query on the given winner
    cell (w_i the factor of grad k'_i: k'_i itself for the RBF kernel, e^{-lambda (r_i - d)} for Matern 3/2)."""
    keys, status, off, mem = model.cells()
    xq = np.asarray(xq, dtype=np.float64)
    out = np.ones(len(xq))
    lam = model.params["lambda"]
    for g in np.unique(cells):
        if g < 0:
            continue
        sel = np.nonzero(cells == g)[0]
        ids = mem[off[g]:off[g + 1]]
        xs = model.x[ids]
        al = model.alpha(int(g))
        r = xq[sel][:, None, :] - xs[None, :, :]
        r2 = np.sum(r * r, axis=2)
        if model.params.get("kernel", 0) in (1, "matern32"):  # gradient weights e^{-lambda (r_i - d)}
            rr = np.sqrt(r2)
            kp = np.exp(-lam * (rr - rr.min(axis=1, keepdims=True)))
        else:  # k'_i = e^{-lambda (r_i^2 - d^2)}
            kp = np.exp(-lam * (r2 - r2.min(axis=1, keepdims=True)))
        num = np.linalg.norm(np.sum((al * kp)[:, :, None] * r, axis=1), axis=1)
        den = np.sum(np.abs(al) * kp * np.sqrt(r2), axis=1)
        out[sel] = num / np.maximum(den, 1e-300)
    return out


def _ang_deg(a, b):
    na = np.linalg.norm(a, axis=1)
    nb = np.linalg.norm(b, axis=1)
    c = np.sum(a * b, axis=1) / np.maximum(na * nb, 1e-300)
    return np.degrees(np.arccos(np.clip(c, -1.0, 1.0)))


def check_mixed(model, xq, sign, gpu, label=""):
    """Assert the mixed-precision GPU outputs (dict of numpy arrays) against the oracle.  Returns stats."""
    xq = np.asarray(xq, dtype=np.float32)
    ref = model.query(xq, sign, with_cands=True)
    gw = gpu["winner"].astype(np.int64)
    rw = ref["winner"].astype(np.int64)
    stats = {"n": len(xq)}
    # SDF: min-fusion is continuous across ties, so it is compared for every query
    err = np.abs(gpu["sdf"].astype(np.float64) - ref["sdf"])
    fin = np.isfinite(ref["sdf"])
    assert np.array_equal(np.isfinite(gpu["sdf"]), fin), label + ": finite pattern differs"
    stats["sdf_max_err"] = float(err[fin].max()) if fin.any() else 0.0
    assert stats["sdf_max_err"] <= SDF_TOL, "%s: max |sdf err| %g" % (label, stats["sdf_max_err"])
    diff = gw != rw
    stats["winner_diff"] = int(diff.sum())
    tie = ((gpu["flags"] | ref["flags"]) & 4) != 0
    stats["near_tie_flagged"] = int(tie.sum())
    unflagged = np.nonzero(diff & ~tie)[0]
    assert unflagged.size == 0, "%s: %d winner disagreements without the near-tie flag, e.g. query %d: gpu %d " \
        "oracle %d, oracle u of the two %s" % (label, unflagged.size, unflagged[0], gw[unflagged[0]], rw[unflagged[0]],
                                              ref["cand_u"][unflagged[0]]) if unflagged.size else ""
    if diff.any():
        # the GPU's winner must be an oracle candidate with u within tolerance of the oracle minimum
        for q in np.nonzero(diff)[0]:
            k = np.nonzero(ref["cand_id"][q] == gw[q])[0]
            assert k.size == 1, "%s: GPU winner %d of query %d is not a candidate" % (label, gw[q], q)
            assert ref["cand_u"][q, k[0]] - np.abs(ref["sdf"][q]) <= SDF_TOL, "%s: query %d winner gap" % (label, q)
        alt = model.eval_cell(xq[diff], gw[diff].astype(np.int32), None if sign is None else sign[diff])
        for key in ("grad", "var_sdf", "var_f"):
            ref[key][diff] = alt[key]
    ok = fin
    # gradient angle with the medial-axis and zero-gradient exclusions only
    ratio = cancellation_ratio(model, xq, np.where(ok, gw, -1))
    zero = ((gpu["flags"] | ref["flags"]) & 8) != 0
    med = ratio < MEDIAL_RATIO
    gsel = ok & ~zero & ~med
    ang = _ang_deg(gpu["grad"].astype(np.float64)[gsel], ref["grad"][gsel])
    stats["angle_max_deg"] = float(ang.max()) if ang.size else 0.0
    stats["medial_excluded"] = int((ok & med).sum())
    if ang.size and stats["angle_max_deg"] > ANGLE_TOL_DEG:
        keys, status, off, mem = model.cells()
        idx = np.nonzero(gsel)[0]
        worst = idx[np.argsort(-ang)[:5]]
        diag = ["q=%d ang=%.3g ratio=%.3g sdf=%.3g N=%d" % (q, a, ratio[q], ref["sdf"][q], off[gw[q] + 1] - off[gw[q]])
                for q, a in zip(worst, np.sort(ang)[::-1][:5])]
        over = ang > ANGLE_TOL_DEG
        diag.append("over=%d of %d; ratio of those: %s" % (over.sum(), ang.size, np.round(ratio[idx[over]], 4)[:12]))
        raise AssertionError("%s: max angle %g deg; %s" % (label, stats["angle_max_deg"], "; ".join(diag)))
    rv = ref["var_sdf"][ok]
    ev = np.abs(gpu["var_sdf"][ok].astype(np.float64) - rv)
    stats["var_sdf_max_rel"] = float(np.max(ev / np.maximum(np.abs(rv), 1e-30))) if ev.size else 0.0
    assert stats["var_sdf_max_rel"] <= VAR_SDF_REL, "%s: var_sdf rel %g" % (label, stats["var_sdf_max_rel"])
    rf = ref["var_f"][ok]
    ef = np.abs(gpu["var_f"][ok].astype(np.float64) - rf)
    stats["var_f_max_scaled"] = float(np.max(ef / np.maximum(rf, VAR_F_FLOOR))) if ef.size else 0.0
    assert stats["var_f_max_scaled"] <= VAR_F_REL, "%s: var_f scaled err %g" % (label, stats["var_f_max_scaled"])
    return stats


def check_f64(model, xq64, sign, gpu, label=""):
    """Assert the plain FP64 GPU outputs against the oracle evaluated at the same binary64 points."""
    ref = model.query_f64(xq64, sign)
    gw = gpu["winner"].astype(np.int64)
    fin = np.isfinite(ref["sdf"])
    stats = {"n": len(xq64)}
    assert np.array_equal(gw, ref["winner"]) or np.all((ref["flags"][gw != ref["winner"]] & 4) != 0), \
        label + ": winner differs outside near ties"
    same = (gw == ref["winner"]) & fin
    scale = np.maximum(np.abs(ref["sdf"]), 1e-3)
    e = np.abs(gpu["sdf"] - ref["sdf"]) / scale
    stats["sdf_max_rel"] = float(e[fin].max()) if fin.any() else 0.0
    assert stats["sdf_max_rel"] <= F64_REL, "%s: sdf rel %g" % (label, stats["sdf_max_rel"])
    ratio = cancellation_ratio(model, xq64, np.where(same, gw, -1))
    gsel = same & (ratio >= MEDIAL_RATIO) & ((ref["flags"] & 8) == 0)
    eg = np.max(np.abs(gpu["grad"] - ref["grad"]), axis=1)
    stats["grad_max_abs"] = float(eg[gsel].max()) if gsel.any() else 0.0
    assert stats["grad_max_abs"] <= F64_REL, "%s: grad abs %g" % (label, stats["grad_max_abs"])
    ev = np.abs(gpu["var_sdf"] - ref["var_sdf"]) / np.maximum(np.abs(ref["var_sdf"]), 1e-30)
    stats["var_sdf_max_rel"] = float(ev[same].max()) if same.any() else 0.0
    assert stats["var_sdf_max_rel"] <= F64_REL, "%s: var_sdf rel %g" % (label, stats["var_sdf_max_rel"])
    ef = np.abs(gpu["var_f"] - ref["var_f"]) / np.maximum(ref["var_f"], 1e-3)
    stats["var_f_max_rel"] = float(ef[same].max()) if same.any() else 0.0
    assert stats["var_f_max_rel"] <= F64_REL, "%s: var_f rel %g" % (label, stats["var_f_max_rel"])
    return stats
