"""GB300-native BFAST Monitor: Python binding of libbfm (include/bfm.h).

Argument marshalling only.  Every step of the per-pixel path (tile staging,
masking, normal equations, solve, residuals, MOSUM, detection) runs in the
library's CUDA kernels.  PyTorch provides device memory and streams.  There
is no CPU path: without the compiled library every call raises.

    import torch, paper_1807_01751_gb300 as bfm
    d = bfm.Design(dates, k=3, f=23.0)                  # bfm_design_create
    out = bfm.monitor(d, Y, n_hist=228, h_frac=0.25, lam=1.69)   # bfm_monitor
    out["break_idx"], out["mean_mosum"], out["sigma"], out["beta"], out["status"]

The C names are exported too (``bfm_design_create``, ``bfm_monitor``,
``bfm_monitor_ex``, ``bfm_monitor_host``, ...), taking raw pointers/ints.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

BFM_F32, BFM_I16 = 0, 1
BFM_ALGO_AUTO, BFM_ALGO_SIMT, BFM_ALGO_MMA, BFM_ALGO_COMPLETE, BFM_ALGO_STREAM, BFM_ALGO_HYBRID = 0, 1, 2, 3, 4, 5
BFM_PX_INCOMPLETE = 5
STATUS_NAMES = {0: "OK", 1: "INSUFFICIENT_HISTORY", 2: "SINGULAR", 3: "DEGENERATE", 4: "NO_MONITOR", 5: "INCOMPLETE",
                255: "TIMEOUT"}
ERRORS = {1: "BFM_EINVAL", 2: "BFM_ENOMEM", 3: "BFM_ECUDA", 4: "BFM_ETIMEOUT", 5: "BFM_EBUSY",
          6: "BFM_EUNSUPPORTED"}

_lock = threading.Lock()
_lib = None


BFM_STATIC_MAX_TILES = 64


class TileSpec(ctypes.Structure):
    """bfm_tile_spec of include/bfm.h (one tile of bfm_batch_run_static)."""
    _fields_ = [("design", ctypes.c_void_p), ("Y", ctypes.c_void_p), ("dtype", ctypes.c_int),
                ("mask_bits", ctypes.c_void_p), ("m", ctypes.c_int64), ("n_hist", ctypes.c_int),
                ("h_frac", ctypes.c_double), ("lam", ctypes.c_double), ("break_idx", ctypes.c_void_p),
                ("mean_mosum", ctypes.c_void_p), ("sigma", ctypes.c_void_p), ("beta", ctypes.c_void_p),
                ("status", ctypes.c_void_p)]


class ServeRequest(ctypes.Structure):
    """bfm_serve_request of include/bfm.h."""
    _fields_ = [("design", ctypes.c_void_p), ("Y", ctypes.c_void_p), ("y_on_host", ctypes.c_int),
                ("dtype", ctypes.c_int), ("mask_bits", ctypes.c_void_p), ("m", ctypes.c_int64),
                ("n_hist", ctypes.c_int), ("h_frac", ctypes.c_double), ("lam", ctypes.c_double),
                ("algo", ctypes.c_int)]


SERVE_STATES = {0: "pending", 1: "running", 2: "done", 3: "failed", 4: "cancelled"}


class BfmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.SO


def load(build_if_missing: bool = True):
    """Load libbfm.so (compiling it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        so = _build.build() if build_if_missing else _build.SO
        if not os.path.exists(so):
            raise RuntimeError(f"libbfm.so not found at {so}; run __graft_entry__.build()")
        lib = ctypes.CDLL(so)
        vp, i32, i64, dbl, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
        lib.bfm_version.restype = ctypes.c_char_p
        lib.bfm_last_error.restype = ctypes.c_char_p
        lib.bfm_max_dates.restype = i32
        lib.bfm_design_create.argtypes = [vp, i32, i32, dbl, ctypes.POINTER(vp)]
        lib.bfm_design_create.restype = i32
        lib.bfm_design_destroy.argtypes = [vp]
        lib.bfm_design_destroy.restype = i32
        lib.bfm_design_K.argtypes = [vp]
        lib.bfm_design_K.restype = i32
        lib.bfm_design_N.argtypes = [vp]
        lib.bfm_design_N.restype = i32
        mon = [vp, vp, i32, vp, i64, i32, dbl, dbl, vp, vp, vp, vp, vp]
        lib.bfm_monitor.argtypes = mon + [vp]
        lib.bfm_monitor.restype = i32
        lib.bfm_monitor_ex.argtypes = mon + [i32, vp]
        lib.bfm_monitor_ex.restype = i32
        lib.bfm_monitor_ext.argtypes = mon + [vp, i32, vp]
        lib.bfm_monitor_ext.restype = i32
        lib.bfm_algo_auto.argtypes = [vp, i32, i32, dbl, vp, i64]
        lib.bfm_algo_auto.restype = i32
        lib.bfm_batch_form.argtypes = [vp, i32, i32, dbl, vp, i64]
        lib.bfm_batch_form.restype = i32
        lib.bfm_lambda.argtypes = [dbl, dbl, dbl, i32, i32, ctypes.c_uint64, ctypes.POINTER(dbl), vp, vp]
        lib.bfm_lambda.restype = i32
        lib.bfm_trace.argtypes = [vp, vp, i32, vp, i64, i32, dbl, vp, i64, vp, vp, vp, vp]
        lib.bfm_trace.restype = i32
        lib.bfm_monitor_host_workspace.argtypes = [vp, i32, i64, i32]
        lib.bfm_monitor_host_workspace.restype = sz
        lib.bfm_monitor_host.argtypes = mon + [vp, sz, i64, vp]
        lib.bfm_monitor_host.restype = i32
        lib.bfm_device_errors.argtypes = [vp, ctypes.POINTER(ctypes.c_uint32)]
        lib.bfm_device_errors.restype = i32
        lib.bfm_stage_wait_limit.argtypes = [ctypes.c_uint64]
        lib.bfm_stage_wait_limit.restype = i32
        lib.bfm_solve_rate.argtypes = [i32, i64, i32, vp, ctypes.POINTER(ctypes.c_float)]
        lib.bfm_solve_rate.restype = i32
        lib.bfm_batch_create.argtypes = [ctypes.POINTER(vp)]
        lib.bfm_batch_create.restype = i32
        lib.bfm_batch_add.argtypes = [vp, vp, vp, i32, vp, i64, i32, dbl, dbl, vp, vp, vp, vp, vp,
                                      ctypes.POINTER(i32)]
        lib.bfm_batch_add.restype = i32
        lib.bfm_batch_run.argtypes = [vp, vp]
        lib.bfm_batch_run.restype = i32
        lib.bfm_batch_autotune.argtypes = [vp, vp, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                           ctypes.POINTER(ctypes.c_float)]
        lib.bfm_batch_autotune.restype = i32
        lib.bfm_batch_set_config.argtypes = [vp, i32, i32]
        lib.bfm_batch_set_config.restype = i32
        lib.bfm_batch_tiles.argtypes = [vp]
        lib.bfm_batch_tiles.restype = i32
        lib.bfm_batch_set_forms.argtypes = [vp, i32]
        lib.bfm_batch_set_forms.restype = i32
        lib.bfm_batch_tile_form.argtypes = [vp, i32]
        lib.bfm_batch_tile_form.restype = i32
        lib.bfm_batch_destroy.argtypes = [vp]
        lib.bfm_batch_destroy.restype = i32
        lib.bfm_batch_run_static.argtypes = [ctypes.POINTER(TileSpec), i32, vp]
        lib.bfm_batch_run_static.restype = i32
        u64 = ctypes.c_uint64
        P = ctypes.POINTER
        lib.bfm_serve_create.argtypes = [sz, i32, P(vp)]
        lib.bfm_serve_submit.argtypes = [vp, P(ServeRequest), P(u64)]
        lib.bfm_serve_poll.argtypes = [vp, u64, P(i32), P(dbl)]
        lib.bfm_serve_result.argtypes = [vp, u64, P(vp), P(vp), P(vp), P(vp), P(vp)]
        lib.bfm_serve_release.argtypes = [vp, u64]
        lib.bfm_serve_cancel.argtypes = [vp, u64]
        lib.bfm_serve_wait_all.argtypes = [vp, dbl]
        lib.bfm_serve_stats.argtypes = [vp, P(dbl), P(dbl), P(i64), P(i64), P(dbl)]
        lib.bfm_serve_destroy.argtypes = [vp]
        for n in ("create", "submit", "poll", "result", "release", "cancel", "wait_all", "stats", "destroy"):
            getattr(lib, "bfm_serve_" + n).restype = i32
        _lib = lib
        return lib


def _check(rc: int):
    if rc != 0:
        raise BfmError(rc, load().bfm_last_error().decode())


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---- C names -----------------------------------------------------------------

def bfm_version() -> str:
    return load().bfm_version().decode()


def bfm_last_error() -> str:
    return load().bfm_last_error().decode()


def bfm_max_dates() -> int:
    return load().bfm_max_dates()


def bfm_design_create(dates, k_harm: int, f: float) -> int:
    import numpy as np
    d = np.ascontiguousarray(dates, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(load().bfm_design_create(d.ctypes.data, int(d.size), int(k_harm), float(f), ctypes.byref(h)))
    return h.value


def bfm_design_destroy(handle: int):
    _check(load().bfm_design_destroy(handle))


def bfm_design_K(handle: int) -> int:
    return load().bfm_design_K(handle)


def bfm_monitor(design, Y, dtype, mask_bits, m, n_hist, h_frac, lam, break_idx, mean_mosum, sigma, beta,
                status, stream=None):
    _check(load().bfm_monitor(int(design), _ptr(Y), int(dtype), _ptr(mask_bits), int(m), int(n_hist),
                              float(h_frac), float(lam), _ptr(break_idx), _ptr(mean_mosum), _ptr(sigma),
                              _ptr(beta), _ptr(status), _stream(stream)))


def bfm_monitor_ex(design, Y, dtype, mask_bits, m, n_hist, h_frac, lam, break_idx, mean_mosum, sigma, beta,
                   status, algo, stream=None):
    _check(load().bfm_monitor_ex(int(design), _ptr(Y), int(dtype), _ptr(mask_bits), int(m), int(n_hist),
                                 float(h_frac), float(lam), _ptr(break_idx), _ptr(mean_mosum), _ptr(sigma),
                                 _ptr(beta), _ptr(status), int(algo), _stream(stream)))


def bfm_lambda(alpha: float, h: float, T: float, G: int = 1000, reps: int = 100000, seed: int = 12345,
               return_stats: bool = False, stream=None):
    """Critical value lambda(alpha, h, T) of Eq. 4 by simulation on the GPU
    (see include/bfm.h); with return_stats also the per-path statistics."""
    import numpy as np
    lam = ctypes.c_double(0.0)
    stats = np.empty(int(reps), dtype=np.float64) if return_stats else None
    _check(load().bfm_lambda(float(alpha), float(h), float(T), int(G), int(reps), ctypes.c_uint64(int(seed)),
                             ctypes.byref(lam), stats.ctypes.data if stats is not None else None, _stream(stream)))
    return (lam.value, stats) if return_stats else lam.value


def bfm_trace(design, Y, dtype, mask_bits, m, n_hist, h_frac, pixels, count, status, mo, resid, stream=None):
    _check(load().bfm_trace(int(design), _ptr(Y), int(dtype), _ptr(mask_bits), int(m), int(n_hist), float(h_frac),
                            _ptr(pixels), int(count), _ptr(status), _ptr(mo), _ptr(resid), _stream(stream)))


def bfm_algo_auto(design, dtype: int, n_hist: int, h_frac: float, Y, m: int) -> int:
    return load().bfm_algo_auto(int(design), int(dtype), int(n_hist), float(h_frac), _ptr(Y), int(m))


def bfm_batch_form(design, dtype: int, n_hist: int, h_frac: float, Y, m: int) -> int:
    return load().bfm_batch_form(int(design), int(dtype), int(n_hist), float(h_frac), _ptr(Y), int(m))


def bfm_monitor_ext(design, Y, dtype, mask_bits, m, n_hist, h_frac, lam, break_idx, mean_mosum, sigma, beta,
                    status, max_mosum, algo, stream=None):
    _check(load().bfm_monitor_ext(int(design), _ptr(Y), int(dtype), _ptr(mask_bits), int(m), int(n_hist),
                                  float(h_frac), float(lam), _ptr(break_idx), _ptr(mean_mosum), _ptr(sigma),
                                  _ptr(beta), _ptr(status), _ptr(max_mosum), int(algo), _stream(stream)))


def bfm_monitor_host_workspace(design, dtype: int, chunk_px: int, with_mask: bool) -> int:
    return load().bfm_monitor_host_workspace(int(design), int(dtype), int(chunk_px), int(bool(with_mask)))


def bfm_monitor_host(design, Y_host, dtype, mask_host, m, n_hist, h_frac, lam, break_idx, mean_mosum, sigma,
                     beta, status, workspace, workspace_bytes, chunk_px, stream=None):
    _check(load().bfm_monitor_host(int(design), _ptr(Y_host), int(dtype), _ptr(mask_host), int(m), int(n_hist),
                                   float(h_frac), float(lam), _ptr(break_idx), _ptr(mean_mosum), _ptr(sigma),
                                   _ptr(beta), _ptr(status), _ptr(workspace), int(workspace_bytes),
                                   int(chunk_px), _stream(stream)))


def bfm_device_errors(stream=None) -> int:
    v = ctypes.c_uint32(0)
    _check(load().bfm_device_errors(_stream(stream), ctypes.byref(v)))
    return v.value


def bfm_solve_rate(K: int, systems: int, fp64: bool, stream=None) -> float:
    """Device ms of two K x K Cholesky solves per system for `systems` systems (FP64 or FP32)."""
    ms = ctypes.c_float(0.0)
    _check(load().bfm_solve_rate(int(K), int(systems), 1 if fp64 else 0, _stream(stream), ctypes.byref(ms)))
    return ms.value


def bfm_stage_wait_limit(consumer_wait_ns: int) -> None:
    """Bound of the streaming form's consumer-side stage waits (0: default 2 s)."""
    _check(load().bfm_stage_wait_limit(int(consumer_wait_ns)))


def bfm_batch_create() -> int:
    h = ctypes.c_void_p()
    _check(load().bfm_batch_create(ctypes.byref(h)))
    return h.value


def bfm_batch_add(batch, design, Y, dtype, mask_bits, m, n_hist, h_frac, lam, break_idx, mean_mosum, sigma, beta,
                  status) -> int:
    tid = ctypes.c_int(-1)
    _check(load().bfm_batch_add(int(batch), int(design), _ptr(Y), int(dtype), _ptr(mask_bits), int(m), int(n_hist),
                                float(h_frac), float(lam), _ptr(break_idx), _ptr(mean_mosum), _ptr(sigma),
                                _ptr(beta), _ptr(status), ctypes.byref(tid)))
    return tid.value


def bfm_batch_run(batch, stream=None):
    _check(load().bfm_batch_run(int(batch), _stream(stream)))


def bfm_batch_autotune(batch, stream=None):
    c, g, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_float(0)
    _check(load().bfm_batch_autotune(int(batch), _stream(stream), ctypes.byref(c), ctypes.byref(g),
                                     ctypes.byref(ms)))
    return c.value, g.value, ms.value


def bfm_batch_set_config(batch, ctas_per_sm: int, grab: int):
    _check(load().bfm_batch_set_config(int(batch), int(ctas_per_sm), int(grab)))


def bfm_batch_set_forms(batch, algo: int):
    _check(load().bfm_batch_set_forms(int(batch), int(algo)))


def bfm_batch_tile_form(batch, tile_id: int) -> int:
    return load().bfm_batch_tile_form(int(batch), int(tile_id))


def bfm_batch_destroy(batch):
    _check(load().bfm_batch_destroy(int(batch)))


def bfm_batch_run_static(specs, stream=None):
    """Run tiles (a list of TileSpec) through bfm_batch_run_static, the entry
    point that allocates no device memory (for callers that cannot allocate
    while they run work: pre-reserved memory pools, latency-critical loops)."""
    arr = (TileSpec * max(1, len(specs)))(*specs)
    _check(load().bfm_batch_run_static(arr, len(specs), _stream(stream)))


def tile_spec(design, Y, *, n_hist: int, h_frac: float, lam: float, out: dict, mask_bits=None) -> TileSpec:
    import torch
    dtype = {torch.float32: BFM_F32, torch.int16: BFM_I16}[Y.dtype]
    return TileSpec(int(design), _ptr(Y), dtype, _ptr(mask_bits), Y.shape[1], int(n_hist), float(h_frac), float(lam),
                    _ptr(out["break_idx"]), _ptr(out["mean_mosum"]), _ptr(out["sigma"]), _ptr(out["beta"]),
                    _ptr(out["status"]))


# ---- convenience layer ----------------------------------------------------------

class Design:
    """Owning wrapper of a bfm_design_t (Algorithm 1, step 1)."""

    def __init__(self, dates, k: int, f: float):
        self.handle = bfm_design_create(dates, k, f)
        self.k = int(k)
        self.K = 2 + 2 * self.k
        self.N = len(dates)
        self.f = float(f)

    def close(self):
        if self.handle:
            bfm_design_destroy(self.handle)
            self.handle = 0

    def __int__(self):
        return int(self.handle)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def empty_outputs(K: int, m: int, device="cuda"):
    import torch
    return dict(break_idx=torch.empty(m, dtype=torch.int32, device=device),
                mean_mosum=torch.empty(m, dtype=torch.float32, device=device),
                sigma=torch.empty(m, dtype=torch.float32, device=device),
                beta=torch.empty((K, m), dtype=torch.float32, device=device),
                status=torch.empty(m, dtype=torch.uint8, device=device))


def monitor(design: Design, Y, *, n_hist: int, h_frac: float, lam: float, mask_bits=None, out=None,
            algo: int = BFM_ALGO_AUTO, stream=None, max_mosum: bool = False):
    """Run bfm_monitor_ex (bfm_monitor_ext with max_mosum=True: one more
    output, "max_mosum") on a device tensor Y [N][m] (float32 or int16)."""
    import torch
    assert Y.is_cuda and Y.dim() == 2 and Y.is_contiguous()
    dtype = {torch.float32: BFM_F32, torch.int16: BFM_I16}[Y.dtype]
    m = Y.shape[1]
    if out is None:
        out = empty_outputs(design.K, m, Y.device)
    if max_mosum:
        if "max_mosum" not in out:
            out["max_mosum"] = torch.empty(m, dtype=torch.float32, device=Y.device)
        bfm_monitor_ext(design, Y, dtype, mask_bits, m, n_hist, h_frac, lam, out["break_idx"], out["mean_mosum"],
                        out["sigma"], out["beta"], out["status"], out["max_mosum"], algo, stream)
    else:
        bfm_monitor_ex(design, Y, dtype, mask_bits, m, n_hist, h_frac, lam, out["break_idx"], out["mean_mosum"],
                       out["sigma"], out["beta"], out["status"], algo, stream)
    return out


def trace(design: Design, Y, *, n_hist: int, h_frac: float, status, pixels=None, count=None, mask_bits=None,
          resid: bool = True, stream=None):
    """bfm_trace on a device tensor Y [N][m]: for the pixels (int64 device
    tensor, or the first `count` pixels) the MOSUM process "mo" and, with
    resid=True, the residuals "resid", each [count][N] float32 indexed by
    the original date (NaN where undefined).  `status` is the status output
    of monitor() on the same data."""
    import torch
    assert Y.is_cuda and Y.dim() == 2 and Y.is_contiguous()
    dtype = {torch.float32: BFM_F32, torch.int16: BFM_I16}[Y.dtype]
    N, m = Y.shape
    if pixels is not None:
        assert pixels.is_cuda and pixels.dtype == torch.int64 and pixels.is_contiguous()
        count = pixels.numel()
    count = int(count)
    out = dict(mo=torch.empty((count, N), dtype=torch.float32, device=Y.device))
    if resid:
        out["resid"] = torch.empty((count, N), dtype=torch.float32, device=Y.device)
    bfm_trace(design, Y, dtype, mask_bits, m, n_hist, h_frac, pixels, count, status, out["mo"], out.get("resid"),
              stream)
    return out


class Batch:
    """Owning wrapper of a bfm_batch_t: tiles added with :meth:`add` run in one
    persistent launch (:meth:`run`), replayed from a CUDA graph."""

    def __init__(self, forms: int = BFM_ALGO_AUTO):
        self.handle = bfm_batch_create()
        self.tiles = []
        self.ids = []
        if forms != BFM_ALGO_AUTO:
            bfm_batch_set_forms(self.handle, forms)

    def add(self, design: Design, Y, *, n_hist: int, h_frac: float, lam: float, mask_bits=None, out=None):
        import torch
        dtype = {torch.float32: BFM_F32, torch.int16: BFM_I16}[Y.dtype]
        m = Y.shape[1]
        if out is None:
            out = empty_outputs(design.K, m, Y.device)
        tid = bfm_batch_add(self.handle, design, Y, dtype, mask_bits, m, n_hist, h_frac, lam, out["break_idx"],
                            out["mean_mosum"], out["sigma"], out["beta"], out["status"])
        self.tiles.append((Y, mask_bits, out))  # keep buffers alive
        self.ids.append(tid)
        return out

    def form(self, i: int) -> int:
        """The form the i-th added tile takes in this batch (BFM_ALGO_*)."""
        return bfm_batch_tile_form(self.handle, self.ids[i])

    def run(self, stream=None):
        bfm_batch_run(self.handle, stream)

    def autotune(self, stream=None):
        return bfm_batch_autotune(self.handle, stream)

    def set_config(self, ctas_per_sm: int, grab: int):
        bfm_batch_set_config(self.handle, ctas_per_sm, grab)

    def close(self):
        if self.handle:
            bfm_batch_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DeviceArray:
    """Minimal __cuda_array_interface__ holder for a library-owned buffer."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


class Server:
    """Owning wrapper of a bfm_server_t (continuous admission under an HBM
    budget; results stay on the device until released)."""

    def __init__(self, hbm_budget: int, slots: int = 4):
        h = ctypes.c_void_p()
        _check(load().bfm_serve_create(int(hbm_budget), int(slots), ctypes.byref(h)))
        self.handle = h.value
        self._keep = {}

    def submit(self, design: Design, Y, *, n_hist: int, h_frac: float, lam: float, mask_bits=None,
               algo: int = BFM_ALGO_AUTO) -> int:
        import torch
        dtype = {torch.float32: BFM_F32, torch.int16: BFM_I16}[Y.dtype]
        req = ServeRequest(int(design), _ptr(Y), int(not Y.is_cuda), dtype, _ptr(mask_bits), int(Y.shape[1]),
                           int(n_hist), float(h_frac), float(lam), int(algo))
        t = ctypes.c_uint64(0)
        _check(load().bfm_serve_submit(self.handle, ctypes.byref(req), ctypes.byref(t)))
        self._keep[t.value] = (design, Y, mask_bits)
        return t.value

    def poll(self, ticket: int):
        st, lat = ctypes.c_int(0), ctypes.c_double(0)
        rc = load().bfm_serve_poll(self.handle, ticket, ctypes.byref(st), ctypes.byref(lat))
        return SERVE_STATES[st.value], lat.value, rc

    def result(self, ticket: int, K: int, m: int, copy: bool = True):
        """The outputs of a done request: zero-copy views of the device-resident
        buffers (valid until release), or copies when `copy`."""
        import torch
        ptrs = [ctypes.c_void_p() for _ in range(5)]
        _check(load().bfm_serve_result(self.handle, ticket, *[ctypes.byref(p) for p in ptrs]))
        spec = [("break_idx", "<i4", (m,)), ("mean_mosum", "<f4", (m,)), ("sigma", "<f4", (m,)),
                ("beta", "<f4", (K, m)), ("status", "|u1", (m,))]
        out = {}
        for (name, ts, shape), p in zip(spec, ptrs):
            v = torch.as_tensor(_DeviceArray(p.value or 0, shape, ts), device="cuda")
            out[name] = v.clone() if copy else v
        return out

    def release(self, ticket: int):
        _check(load().bfm_serve_release(self.handle, ticket))
        self._keep.pop(ticket, None)

    def cancel(self, ticket: int):
        _check(load().bfm_serve_cancel(self.handle, ticket))

    def wait_all(self, timeout_s: float = 60.0):
        _check(load().bfm_serve_wait_all(self.handle, float(timeout_s)))

    def stats(self):
        p50, p99, span = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
        n, px = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(load().bfm_serve_stats(self.handle, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(n),
                                      ctypes.byref(px), ctypes.byref(span)))
        return dict(p50_ms=p50.value, p99_ms=p99.value, completed=n.value, pixels=px.value, span_ms=span.value)

    def close(self):
        if self.handle:
            _check(load().bfm_serve_destroy(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
