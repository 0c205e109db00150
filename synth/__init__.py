"""Seeded synthetic BFAST Monitor workloads (inputs only, no method arithmetic).

The scenes stand in for the paper's Landsat data (Section 4.3), which is not
available here: NDVI-like season-trend series on a 16-day revisit with date
jitter, cloud gaps (i.i.d. or a two-state Markov chain) and injected level
shifts in the monitoring period, stored time-major as Y[N][m] (Section 3,
Eq. 7).  Generation runs in C (``synth.c``) with one SplitMix64 stream per
pixel, so a scene is the same whatever the thread count.

Named workloads:
  * ``c1``  m=4096, N=228, n_hist=100, k=3 (K=8), f=23, h=0.25, i.i.d. 30 %
    missing, 20 % of pixels with a -0.3 shift; y = 0.5 + 0.001 t
    + 0.2 sin(2 pi t/f) + 0.05 cos(4 pi t/f) + N(0, 0.03).  float32, seed 1.
  * ``c2``  m=8,388,608 (4096 x 2048), N=414, n_hist=228, K=8, f=23, h=0.25,
    intercept 0.5, six harmonic coefficients ~ U(0, 0.3), noise N(0, 0.04),
    Markov clouds (~60 % missing, mean run 4), 10 % of pixels with a shift
    ~ U(-0.5, -0.1).  float32, seed 2.
  * ``c3``  the c1 scene stored as int16 NDVI*1e4 (-32768 = missing).
  * ``c4``  64 uneven int16 tiles (see :func:`tiles_c4`).

The critical value lambda of each workload comes from ``lambda_table.json``,
written by ``synth/make_lambda_table.py`` (Monte-Carlo of the limiting MOSUM
process, alpha = 0.05).
"""
from __future__ import annotations

import ctypes
import json
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile synth.c into a shared library (gcc, OpenMP)."""
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
            lib.synth_dates.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p]
            lib.synth_dates.restype = None
            lib.synth_scene.argtypes = [
                ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_double,
                ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                ctypes.c_void_p]
            lib.synth_scene.restype = None
            _lib = lib
    return _lib


def dates(seed: int, N: int) -> np.ndarray:
    """t_i = (16 i + U{-3..3}) / 16, i = 1..N (16-day revisit with jitter)."""
    out = np.empty(N, dtype=np.float64)
    _load().synth_dates(ctypes.c_uint64(seed), N, out.ctypes.data)
    return out


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data if isinstance(a, np.ndarray) else int(a))


def scene(*, seed: int, m: int, N: int, n_hist: int, f: float = 23.0, k_gen: int = 3,
          intercept: float = 0.5, slope: float = 0.0, coef_fixed=None, coef_umax: float = 0.3,
          noise_sd: float = 0.04, miss: str = "markov", p_a: float = 0.25, p_b: float = 0.375,
          break_frac: float = 0.1, step=(-0.5, -0.1), dtype: str = "f32", date_vals=None,
          out_ptr: int | None = None):
    """Generate one scene.  Returns (dates, Y, true_break).

    ``miss``: "none", "iid" (probability p_a) or "markov" (P(missing->clear)
    = p_a, P(clear->missing) = p_b).  ``dtype`` "f32" (NaN = missing) or "i16"
    (round(y*1e4), -32768 = missing).  ``out_ptr`` lets the caller supply the
    [N][m] buffer (e.g. pinned host memory); Y is then returned as None.
    """
    lib = _load()
    d = dates(seed, N) if date_vals is None else np.ascontiguousarray(date_vals, dtype=np.float64)
    mk = {"none": 0, "iid": 1, "markov": 2}[miss]
    cf = None if coef_fixed is None else np.ascontiguousarray(coef_fixed, dtype=np.float64)
    if cf is not None:
        assert cf.size == 2 * k_gen
    brk = np.empty(m, dtype=np.int32)
    Y = None
    if out_ptr is None:
        Y = np.empty((N, m), dtype=np.float32 if dtype == "f32" else np.int16)
        ptr = Y.ctypes.data
    else:
        ptr = out_ptr
    yf = ctypes.c_void_p(ptr) if dtype == "f32" else None
    yi = ctypes.c_void_p(ptr) if dtype == "i16" else None
    lib.synth_scene(ctypes.c_uint64(seed), m, N, d.ctypes.data, f, n_hist, k_gen, intercept, slope,
                    _ptr(cf), coef_umax, noise_sd, mk, p_a, p_b, break_frac, float(step[0]),
                    float(step[1]), yf, yi, brk.ctypes.data)
    return d, Y, brk


def lambda_table() -> dict:
    with open(os.path.join(_HERE, "lambda_table.json")) as fh:
        return json.load(fh)


def workload_lambda(name: str) -> float:
    return float(lambda_table()["workloads"][name]["lambda"])


WORKLOADS = {
    "c1": dict(seed=1, m=4096, N=228, n_hist=100, f=23.0, k=3, h_frac=0.25, dtype="f32",
               gen=dict(k_gen=2, intercept=0.5, slope=0.001, coef_fixed=[0.2, 0.0, 0.0, 0.05],
                        noise_sd=0.03, miss="iid", p_a=0.3, break_frac=0.2, step=(-0.3, -0.3))),
    "c2": dict(seed=2, m=8388608, N=414, n_hist=228, f=23.0, k=3, h_frac=0.25, dtype="f32",
               gen=dict(k_gen=3, intercept=0.5, slope=0.0, coef_umax=0.3, noise_sd=0.04,
                        miss="markov", p_a=0.25, p_b=0.375, break_frac=0.1, step=(-0.5, -0.1))),
    # the c2 scene without clouds (series with no missing value: the shared pseudo-inverse form)
    "c2_complete": dict(seed=2, m=8388608, N=414, n_hist=228, f=23.0, k=3, h_frac=0.25, dtype="f32", lam_of="c2",
                        gen=dict(k_gen=3, intercept=0.5, slope=0.0, coef_umax=0.3, noise_sd=0.04,
                                 miss="none", break_frac=0.1, step=(-0.5, -0.1))),
    "c3": dict(seed=1, m=4096, N=228, n_hist=100, f=23.0, k=3, h_frac=0.25, dtype="i16",
               gen=dict(k_gen=2, intercept=0.5, slope=0.001, coef_fixed=[0.2, 0.0, 0.0, 0.05],
                        noise_sd=0.03, miss="iid", p_a=0.3, break_frac=0.2, step=(-0.3, -0.3))),
}


def workload(name: str, *, m: int | None = None, out_ptr: int | None = None, dtype: str | None = None):
    """Generate a named workload (optionally with fewer pixels m: the first m
    pixels of the same scene, since every pixel has its own stream).  Returns
    a dict with dates, Y, true_break and the monitoring parameters."""
    w = WORKLOADS[name]
    mm = w["m"] if m is None else int(m)
    dt = w["dtype"] if dtype is None else dtype
    d, Y, brk = scene(seed=w["seed"], m=mm, N=w["N"], n_hist=w["n_hist"], f=w["f"], dtype=dt,
                      out_ptr=out_ptr, **w["gen"])
    return dict(name=name, dates=d, Y=Y, true_break=brk, m=mm, N=w["N"], n_hist=w["n_hist"],
                f=w["f"], k=w["k"], h_frac=w["h_frac"], lam=workload_lambda(w.get("lam_of", name)), dtype=dt)


def tiles_c4(seed: int = 4, count: int = 64, scale: float = 1.0, px_multiple: int = 1):
    """Parameters of the uneven-tile batch: pixels log-U[1e4, 2e6] (times
    ``scale``), N ~ U{120..600}, k ~ U{1..3}, history fraction U(0.4, 0.7),
    missing fraction U(0.2, 0.7) as a Markov chain with mean missing run 4
    (P(missing->clear) = 0.25), int16 storage, h = 0.25.  ``px_multiple``
    rounds the pixel counts up (8: int16 rows of whole 16-byte units)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        m = int(round(math.exp(rng.uniform(math.log(1e4), math.log(2e6))) * scale))
        m = -(-m // px_multiple) * px_multiple
        N = int(rng.integers(120, 601))
        k = int(rng.integers(1, 4))
        hf = float(rng.uniform(0.4, 0.7))
        miss = float(rng.uniform(0.2, 0.7))
        p_a = 0.25
        p_b = miss * p_a / (1.0 - miss)
        out.append(dict(tile=i, seed=1000 + i, m=max(m, 1), N=N, k=k, n_hist=max(int(hf * N), 2 * k + 3),
                        miss=miss, p_a=p_a, p_b=p_b, h_frac=0.25, f=23.0))
    return out


# ---- device-side generation of large scenes ---------------------------------------
#
# The full c2 scene (8.4 M pixels x 414 dates) takes minutes through the C
# generator, so large scenes are drawn on the GPU with PyTorch's seeded
# generator instead: the same recipe (dates, signal, noise, cloud chain,
# shifts), different random streams.  Tests that check such a scene against
# the oracle copy the sampled pixel columns back from the device.

_TORCH_CHUNK = 1 << 22


def scene_torch(*, seed: int, m: int, N: int, n_hist: int, f: float = 23.0, k_gen: int = 3,
                intercept: float = 0.5, slope: float = 0.0, coef_fixed=None, coef_umax: float = 0.3,
                noise_sd: float = 0.04, miss: str = "markov", p_a: float = 0.25, p_b: float = 0.375,
                break_frac: float = 0.1, step=(-0.5, -0.1), dtype: str = "f32", device="cuda",
                date_vals=None):
    """Generate a scene directly in device memory.  Returns (dates numpy,
    Y [N][m] tensor, true_break [m] int32 tensor).  Deterministic for a given
    (seed, m): pixel chunks of 2^22 get their own generator seed."""
    import torch
    d = dates(seed, N) if date_vals is None else np.ascontiguousarray(date_vals, dtype=np.float64)
    tt = np.asarray(d)
    harm = np.empty((N, 2 * k_gen))
    for j in range(1, k_gen + 1):
        harm[:, 2 * (j - 1)] = np.sin(2 * np.pi * j * tt / f)
        harm[:, 2 * (j - 1) + 1] = np.cos(2 * np.pi * j * tt / f)
    harm_t = torch.from_numpy(harm.astype(np.float32)).to(device)
    base_t = torch.from_numpy((intercept + slope * tt).astype(np.float32)).to(device)
    tdtype = torch.float32 if dtype == "f32" else torch.int16
    Y = torch.empty((N, m), dtype=tdtype, device=device)
    brk = torch.empty(m, dtype=torch.int32, device=device)
    pi_miss = p_b / (p_a + p_b) if (p_a + p_b) > 0 else 0.0
    for ci, c0 in enumerate(range(0, m, _TORCH_CHUNK)):
        mc = min(_TORCH_CHUNK, m - c0)
        g = torch.Generator(device=device)
        g.manual_seed((seed * 1000003 + ci * 7919 + 17) % (2**63 - 1))
        if coef_fixed is not None:
            coef = torch.tensor(coef_fixed, dtype=torch.float32, device=device).expand(mc, 2 * k_gen)
        else:
            coef = torch.rand((mc, 2 * k_gen), generator=g, device=device) * coef_umax
        is_b = torch.rand(mc, generator=g, device=device) < break_frac
        span = N - n_hist
        bd = n_hist + torch.floor(torch.rand(mc, generator=g, device=device) * span).to(torch.int32)
        bd = torch.clamp(bd, max=N - 1)
        stp = step[0] + (step[1] - step[0]) * torch.rand(mc, generator=g, device=device)
        bdate = torch.where(is_b & (span > 0), bd, torch.full_like(bd, -1))
        brk[c0:c0 + mc] = bdate
        state = torch.rand(mc, generator=g, device=device) < pi_miss if miss == "markov" else None
        sig = coef @ harm_t.T  # [mc, N]
        for t in range(N):
            if miss == "markov":
                if t > 0:
                    u = torch.rand(mc, generator=g, device=device)
                    state = torch.where(state, ~(u < p_a), u < p_b)
                mt = state
            elif miss == "iid":
                mt = torch.rand(mc, generator=g, device=device) < p_a
            else:
                mt = None
            y = base_t[t] + sig[:, t] + noise_sd * torch.randn(mc, generator=g, device=device)
            y = y + torch.where((bdate >= 0) & (t >= bdate), stp, torch.zeros_like(stp))
            if dtype == "f32":
                if mt is not None:
                    y = torch.where(mt, torch.full_like(y, float("nan")), y)
                Y[t, c0:c0 + mc] = y
            else:
                v = torch.clamp(torch.round(y * 1e4), -32767, 32767).to(torch.int16)
                if mt is not None:
                    v = torch.where(mt, torch.full_like(v, -32768), v)
                Y[t, c0:c0 + mc] = v
        del sig
    return d, Y, brk


def workload_torch(name: str, *, m: int | None = None, device="cuda", dtype: str | None = None):
    """Device-resident version of :func:`workload` (same recipe, torch streams)."""
    w = WORKLOADS[name]
    mm = w["m"] if m is None else int(m)
    dt = w["dtype"] if dtype is None else dtype
    d, Y, brk = scene_torch(seed=w["seed"], m=mm, N=w["N"], n_hist=w["n_hist"], f=w["f"], dtype=dt,
                            device=device, **w["gen"])
    return dict(name=name, dates=d, Y=Y, true_break=brk, m=mm, N=w["N"], n_hist=w["n_hist"], f=w["f"],
                k=w["k"], h_frac=w["h_frac"], lam=workload_lambda(w.get("lam_of", name)), dtype=dt)


def lambda_for_horizon(T: float) -> float:
    """lambda at alpha = 0.05, h = 0.25 for horizon T = N/n, linearly
    interpolated in the stored grid (T in [1.2, 3.0], clamped)."""
    grid = lambda_table()["grid_h0.25_alpha0.05"]
    xs = sorted(float(k) for k in grid)
    ys = [grid[f"{x:.1f}"] for x in xs]
    return float(np.interp(min(max(T, xs[0]), xs[-1]), xs, ys))
