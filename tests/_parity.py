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
