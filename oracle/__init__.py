"""FP64 oracle for the BFAST Monitor per-pixel path.

TEST INFRASTRUCTURE ONLY: the plain, slow reference that the CUDA path is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it.  It shares no code with the CUDA
library (``paper_1807_01751_gb300``) and imports nothing from it.

The arithmetic lives in ``bfm_oracle.c`` (plain C, double precision, OpenMP
over pixels); this module compiles it with gcc and wraps it with ctypes.  See
the header of ``bfm_oracle.c`` for the definition it follows (Section 2.1,
Eq. 1-6, Algorithm 1) and the readings taken where the paper is silent.

Parity pins (what ties the oracle to the paper and to mathematics rather than
to itself) live in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bfm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "OK", 1: "INSUFFICIENT_HISTORY", 2: "SINGULAR", 3: "DEGENERATE", 4: "NO_MONITOR"}


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
            lib.oracle_design.argtypes = [vp, i32, i32, dbl, vp]
            lib.oracle_design.restype = None
            lib.oracle_lstsq_qr.argtypes = [i32, i32, vp, vp, vp, vp]
            lib.oracle_lstsq_qr.restype = i32
            lib.oracle_lstsq_normal.argtypes = [i32, i32, vp, vp, vp]
            lib.oracle_lstsq_normal.restype = i32
            lib.oracle_logplus.argtypes = [dbl]
            lib.oracle_logplus.restype = dbl
            lib.oracle_boundary.argtypes = [dbl, i32, i32]
            lib.oracle_boundary.restype = dbl
            lib.oracle_monitor.argtypes = [i64, i32, vp, i32, dbl, vp, vp, i32, dbl, dbl,
                                           vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
            lib.oracle_monitor.restype = None
            lib.oracle_lambda.argtypes = [dbl, dbl, dbl, i32, i32, ctypes.c_uint64, vp]
            lib.oracle_lambda.restype = dbl
            _lib = lib
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def design(dates, k: int, f: float) -> np.ndarray:
    """X with rows x_t of Eq. 2 (raw date values), shape [N, 2+2k]."""
    d = _c(dates, np.float64)
    X = np.empty((d.size, 2 + 2 * k), dtype=np.float64)
    _load().oracle_design(d.ctypes.data, d.size, k, f, X.ctypes.data)
    return X


def lstsq_qr(A, y):
    """Householder-QR least squares; returns (beta, diag(R))."""
    A = _c(A, np.float64).copy()
    y = _c(y, np.float64).copy()
    n, K = A.shape
    beta = np.empty(K)
    rd = np.empty(K)
    _load().oracle_lstsq_qr(n, K, A.ctypes.data, y.ctypes.data, beta.ctypes.data, rd.ctypes.data)
    return beta, rd


def lstsq_normal(A, y):
    """Normal-equation (Eq. 6) least squares by Cholesky; returns beta."""
    A = _c(A, np.float64)
    y = _c(y, np.float64)
    n, K = A.shape
    beta = np.empty(K)
    rc = _load().oracle_lstsq_normal(n, K, A.ctypes.data, y.ctypes.data, beta.ctypes.data)
    if rc:
        beta[:] = np.nan
    return beta


def logplus(x: float) -> float:
    return _load().oracle_logplus(float(x))


def boundary(lam: float, j: int, n: int) -> float:
    return _load().oracle_boundary(float(lam), int(j), int(n))


def valid_and_values(Y, mask_bits=None):
    """Missing-value convention shared by the public API: float NaN or int16
    -32768 is missing; an optional bit mask [N][ceil(m/32)] (bit p%32 of word
    p//32, 1 = valid) is ANDed in.  Returns (values as float64, valid uint8)."""
    Y = np.asarray(Y)
    if Y.dtype == np.int16:
        valid = Y != np.int16(-32768)
    else:
        valid = ~np.isnan(Y)
    vals = np.where(valid, Y.astype(np.float64), 0.0)
    if mask_bits is not None:
        N, m = Y.shape
        mb = np.asarray(mask_bits, dtype=np.uint32)
        p = np.arange(m)
        bits = (mb[:, p // 32] >> (p % 32).astype(np.uint32)) & np.uint32(1)
        valid = valid & (bits == 1)
    return vals, valid.astype(np.uint8)


def monitor(dates, Y, *, k: int, f: float, n_hist: int, h_frac: float, lam: float,
            mask_bits=None, trace: bool = False) -> dict:
    """Run the oracle on Y [N][m] (float32/float64 with NaN, or int16 with
    -32768, as stored).  Returns a dict of numpy arrays: break_idx, mean_mosum,
    sigma, beta [K][m], status, n, Nv, h, margin (and mo_trace [m][N])."""
    d = _c(dates, np.float64)
    vals, valid = valid_and_values(Y, mask_bits)
    vals = np.ascontiguousarray(vals)
    valid = np.ascontiguousarray(valid)
    N, m = vals.shape
    K = 2 + 2 * k
    out = dict(
        break_idx=np.empty(m, np.int32), mean_mosum=np.empty(m), sigma=np.empty(m),
        beta=np.empty((K, m)), status=np.empty(m, np.uint8), n=np.empty(m, np.int32),
        Nv=np.empty(m, np.int32), h=np.empty(m, np.int32), margin=np.empty(m))
    tr = np.empty((m, N)) if trace else None
    _load().oracle_monitor(m, N, d.ctypes.data, k, f, vals.ctypes.data, valid.ctypes.data, n_hist,
                           h_frac, lam, out["break_idx"].ctypes.data, out["mean_mosum"].ctypes.data,
                           out["sigma"].ctypes.data, out["beta"].ctypes.data,
                           out["status"].ctypes.data, out["n"].ctypes.data, out["Nv"].ctypes.data,
                           out["h"].ctypes.data, out["margin"].ctypes.data,
                           None if tr is None else tr.ctypes.data)
    if trace:
        out["mo_trace"] = tr
    return out


def max_mosum(out: dict) -> np.ndarray:
    """From monitor(..., trace=True): per pixel the MO of largest magnitude
    over the monitoring positions (signed, the first of equal magnitudes), 0
    for DEGENERATE, NaN for pixels without a fit or without monitoring data
    (the map of maximum absolute MOSUM values, Section 4.3)."""
    tr = out["mo_trace"]
    m = tr.shape[0]
    res = np.full(m, np.nan)
    for p in range(m):
        st = out["status"][p]
        if st == 3:
            res[p] = 0.0
        elif st == 0:
            row = tr[p][~np.isnan(tr[p])]
            res[p] = row[int(np.argmax(np.abs(row)))]
    return res


def critical_value(alpha: float, h: float, T: float, *, G: int = 1000, reps: int = 100000,
                   seed: int = 12345, return_stats: bool = False):
    """lambda(alpha, h, T) as the (1-alpha) quantile of the simulated supremum
    of |W(t) - W(t-h) - h W(1)| / sqrt(log+ t) over t in [1, T]."""
    stats = np.empty(reps)
    lam = _load().oracle_lambda(alpha, h, T, G, reps, ctypes.c_uint64(seed), stats.ctypes.data)
    return (lam, stats) if return_stats else lam
