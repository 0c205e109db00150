"""Comparison of CUDA-path outputs with the FP64 oracle, element by element.

Tolerances (stated per output, for the float path):
  * break_idx: equal, except on margin-tied pixels, i.e. where the oracle's
    min_j ||MO_j| - b_j| up to its break is below 1e-5 (counted, reported);
  * beta: column-scaled error max_i |dbeta_i| ||X_i||_inf / max_i |beta_i|
    ||X_i||_inf (the trend coefficient is ~1e-3, so a plain relative error
    on it is ill-posed);
  * sigma: relative error;
  * mean MOSUM: |d| <= tol * max(1, |ref|) (MO is in normalised units);
  * status: equal.
"""
from __future__ import annotations

import numpy as np

import oracle

MARGIN_TIE = 1e-5


def compare(gpu: dict, ref: dict, dates, k: int, f: float, *, tol: float, margin_tie: float = MARGIN_TIE,
            strict_status: bool = True) -> dict:
    st_g = np.asarray(gpu["status"])
    st_r = np.asarray(ref["status"])
    rep = {"pixels": int(st_r.size)}
    st_mis = st_g != st_r
    rep["status_mismatch"] = int(st_mis.sum())
    same = ~st_mis
    tie = np.asarray(ref["margin"]) < margin_tie
    bg, br = np.asarray(gpu["break_idx"]), np.asarray(ref["break_idx"])
    bmis = (bg != br) & same
    rep["margin_tied"] = int(tie.sum())
    rep["break_mismatch_tied"] = int((bmis & tie).sum())
    rep["break_mismatch_untied"] = int((bmis & ~tie).sum())
    X = oracle.design(dates, k, f)
    colmax = np.abs(X).max(axis=0)[:, None]
    fitted = same & np.isin(st_r, [0, 3, 4])
    bgm, brm = np.asarray(gpu["beta"], np.float64), np.asarray(ref["beta"])
    if fitted.any():
        num = np.max(np.abs(bgm[:, fitted] - brm[:, fitted]) * colmax, axis=0)
        den = np.max(np.abs(brm[:, fitted]) * colmax, axis=0)
        be = num / np.maximum(den, 1e-300)
        rep["beta_err_max"] = float(be.max())
        rep["beta_err_p99"] = float(np.quantile(be, 0.99))
    else:
        rep["beta_err_max"] = 0.0
    sig_ok = same & np.isin(st_r, [0, 4])
    if sig_ok.any():
        se = np.abs(np.asarray(gpu["sigma"], np.float64)[sig_ok] - ref["sigma"][sig_ok]) / ref["sigma"][sig_ok]
        rep["sigma_err_max"] = float(se.max())
    else:
        rep["sigma_err_max"] = 0.0
    mo_ok = same & (st_r == 0)
    if mo_ok.any():
        rm = ref["mean_mosum"][mo_ok]
        me = np.abs(np.asarray(gpu["mean_mosum"], np.float64)[mo_ok] - rm) / np.maximum(1.0, np.abs(rm))
        rep["mean_err_max"] = float(me.max())
    else:
        rep["mean_err_max"] = 0.0
    # NaN conventions of the unfitted statuses
    nf = same & np.isin(st_r, [1, 2])
    rep["nan_convention_ok"] = bool(np.isnan(np.asarray(gpu["beta"])[:, nf]).all()
                                    and np.isnan(np.asarray(gpu["sigma"])[nf]).all()
                                    and (bg[nf] == -1).all())
    nm = same & (st_r == 4)
    rep["no_monitor_ok"] = bool(np.isnan(np.asarray(gpu["mean_mosum"])[nm]).all() and (bg[nm] == -1).all())
    dg = same & (st_r == 3)
    rep["degenerate_ok"] = bool((np.asarray(gpu["mean_mosum"])[dg] == 0).all() and (bg[dg] == -1).all())
    rep["ok"] = bool((rep["status_mismatch"] == 0 or not strict_status)
                     and rep["break_mismatch_untied"] == 0
                     and rep["beta_err_max"] <= tol and rep["sigma_err_max"] <= tol
                     and rep["mean_err_max"] <= tol and rep["nan_convention_ok"] and rep["no_monitor_ok"]
                     and rep["degenerate_ok"])
    return rep


def to_numpy(out: dict) -> dict:
    return {k: v.cpu().numpy() for k, v in out.items()}


EPS_OUT = 2.0 ** -23  # two roundings to float


def check_trace_rows(sel, mo, rs, ref, vals, valid, X, lam, *, m):
    """bfm_trace rows (mo, rs: [len(sel)][N]; rs may be None) against the
    oracle's results (ref from oracle.monitor(..., trace=True) plus
    ref["n_hist"]; vals/valid from oracle.valid_and_values; X the raw Eq. 2
    design) for the pixels `sel`, indices into ref's pixels (outside 0..m-1:
    rows of NaN).  MO by monitoring position is mapped to the original dates;
    reference residuals are y - x'beta with the oracle's beta.  Tolerance: the
    float rounding of the output plus 1e-9 relative (both sides FP64).
    Returns (worst MO error, worst residual error / max|y|, breaks checked)."""
    worst_mo = worst_r = 0.0
    checked_breaks = 0
    for row, p in enumerate(sel):
        if p < 0 or p >= m:
            assert np.isnan(mo[row]).all() and (rs is None or np.isnan(rs[row]).all())
            continue
        st = ref["status"][p]
        if st in (1, 2):
            assert np.isnan(mo[row]).all() and (rs is None or np.isnan(rs[row]).all())
            continue
        idx = np.nonzero(valid[:, p])[0]
        n_p = int(ref["n"][p])
        assert n_p == (idx < ref["n_hist"]).sum()
        if rs is not None:
            r_ref = vals[idx, p] - X[idx] @ ref["beta"][:, p]
            assert np.isnan(np.delete(rs[row], idx)).all()
            ymax = np.abs(vals[idx[:n_p], p]).max()
            d = np.abs(rs[row, idx].astype(np.float64) - r_ref)
            assert (d <= 1e-9 * ymax + EPS_OUT * np.abs(r_ref)).all(), (p, d.max())
            worst_r = max(worst_r, d.max() / max(ymax, 1e-30))
        mon = idx[n_p:]
        assert np.isnan(np.delete(mo[row], mon)).all()
        g = mo[row, mon].astype(np.float64)
        if st == 3:
            assert (g == 0).all()
            continue
        if st == 4:
            assert mon.size == 0
            continue
        tr = ref["mo_trace"][p][: mon.size]
        d = np.abs(g - tr)
        assert (d <= 1e-9 * np.maximum(1.0, np.abs(tr)) + EPS_OUT * np.abs(tr)).all(), (p, d.max())
        worst_mo = max(worst_mo, (d / np.maximum(1.0, np.abs(tr))).max())
        # the trace crosses the boundary first where bfm_monitor/the oracle put the break
        if ref["margin"][p] > 1e-5:
            j = np.arange(n_p + 1, n_p + 1 + mon.size)
            b = np.array([oracle.boundary(lam, int(jj), n_p) for jj in j])
            cross = np.nonzero(np.abs(g) > b)[0]
            first = mon[cross[0]] if cross.size else -1
            assert first == ref["break_idx"][p], (p, first, ref["break_idx"][p])
            checked_breaks += 1
    return worst_mo, worst_r, checked_breaks
