"""CUDA path vs FP64 oracle, element by element, through the C ABI, in the
four general forms (CUDA-core, tensor-core, streaming CUDA-core, hybrid) on
float storage.

Float path tolerance 1e-5 (beta column-scaled, sigma relative, mean MOSUM
relative to max(1, |ref|)); break indices equal except on margin-tied pixels.
"""
import numpy as np
import pytest

import oracle
import synth
from _parity import check_trace_rows, compare, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5


@pytest.fixture(scope="module")
def bfm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_01751_gb300 as bfm
    bfm.load()
    return bfm


def _run(bfm, w, Y, *, mask=None, algo=0, k=None):
    k = w["k"] if k is None else k
    d = bfm.Design(w["dates"], k, w["f"])
    Yd = torch.from_numpy(np.ascontiguousarray(Y)).cuda()
    md = None if mask is None else torch.from_numpy(mask.view(np.int32)).cuda()
    out = bfm.monitor(d, Yd, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"], mask_bits=md, algo=algo)
    torch.cuda.synchronize()
    assert bfm.bfm_device_errors() == 0
    return to_numpy(out)


def _check(w, Y, gpu, *, k=None, mask=None, tol=TOL_F32):
    k = w["k"] if k is None else k
    ref = oracle.monitor(w["dates"], Y, k=k, f=w["f"], n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"],
                         mask_bits=mask)
    rep = compare(gpu, ref, w["dates"], k, w["f"], tol=tol)
    print(rep)
    assert rep["ok"], rep
    return rep, ref


ALGOS = pytest.mark.parametrize("algo", [1, 2, 4, 5], ids=["simt", "mma", "stream", "hybrid"])


@ALGOS
def test_c1_full_tma(bfm, algo):
    """c1 (m=4096, N=228, K=8, 30 % NaN): 128 tiles of 32 pixels, TMA loader."""
    w = synth.workload("c1")
    gpu = _run(bfm, w, w["Y"], algo=algo)
    rep, ref = _check(w, w["Y"], gpu)
    assert (ref["break_idx"] >= 0).sum() > 500


@pytest.mark.parametrize("algo", [0, 1], ids=["auto", "simt"])
@pytest.mark.parametrize("m", [1, 31, 33, 129, 4093])
def test_c1_ragged_plain_loader(bfm, m, algo):
    """m not a multiple of 4 (or < 32) takes the plain-load tile loader of the
    CUDA-core form (AUTO picks it: the tensor-core form needs a TMA-describable
    Y); the last tile is ragged."""
    w = synth.workload("c1", m=m)
    gpu = _run(bfm, w, w["Y"], algo=algo)
    _check(w, w["Y"], gpu)


@ALGOS
def test_c1_ragged_tma_tail(bfm, algo):
    """m = 4100: TMA loader, last tile has 4 live pixels (out-of-range box
    columns are zero-filled and must not be written)."""
    w = synth.workload("c1", m=4100)
    gpu = _run(bfm, w, w["Y"], algo=algo)
    _check(w, w["Y"], gpu)


@ALGOS
def test_c1_mask_bits(bfm, algo):
    w = synth.workload("c1", m=1000)
    rng = np.random.default_rng(3)
    words = (1000 + 31) // 32
    mask = (rng.random((w["N"], words * 32)) > 0.2)
    bits = np.zeros((w["N"], words), np.uint32)
    for b in range(32):
        bits |= (mask[:, b::32].astype(np.uint32) << np.uint32(b))
    gpu = _run(bfm, w, w["Y"], mask=bits, algo=algo)
    _check(w, w["Y"], gpu, mask=bits)


@pytest.mark.parametrize("algo", [1, 4, 5], ids=["simt", "stream", "hybrid"])
def test_c3_int16_simt(bfm, algo):
    """int16 storage (NDVI*1e4, -32768 missing) on the CUDA-core paths."""
    w = synth.workload("c3")
    gpu = _run(bfm, w, w["Y"], algo=algo)
    _check(w, w["Y"], gpu)


@ALGOS
@pytest.mark.parametrize("k", [1, 2])
def test_fewer_harmonics(bfm, k, algo):
    w = synth.workload("c1", m=2048)
    d, Y, _ = synth.scene(seed=21 + k, m=2048, N=w["N"], n_hist=w["n_hist"], f=23.0, k_gen=k, intercept=0.4,
                          slope=0.0005, coef_umax=0.2, noise_sd=0.02, miss="markov", p_a=0.3, p_b=0.3,
                          break_frac=0.2, step=(-0.4, -0.1))
    w2 = dict(w, dates=d)
    gpu = _run(bfm, w2, Y, k=k, algo=algo)
    _check(w2, Y, gpu, k=k)


@ALGOS
def test_edge_statuses(bfm, algo):
    """Pixels crafted for every status, placed on tile boundaries (lanes 0,
    31, 32, 63): all missing, too few history obs, no monitoring data,
    noise-free (degenerate), collinear history (singular)."""
    w = synth.workload("c1", m=128 if algo == 2 else 96)
    Y = w["Y"].copy()
    N, n = w["N"], w["n_hist"]
    Y[:, 0] = np.nan
    Y[8:n, 31] = np.nan
    Y[n:, 32] = np.nan
    d = w["dates"]
    X = oracle.design(d, 3, 23.0)
    Y[:, 63] = (X @ np.array([0.5, 0.001, 0.2, 0.0, 0.0, 0.05, 0.0, 0.0])).astype(np.float32)
    keep = np.zeros(N, bool)
    keep[np.arange(0, N, 23)] = True
    Y[~keep, 64] = np.nan
    gpu = _run(bfm, w, Y, algo=algo)
    rep, ref = _check(w, Y, gpu)
    assert ref["status"][0] == 1 and ref["status"][31] == 1 and ref["status"][32] == 4
    assert ref["status"][63] == 3 and ref["status"][64] in (1, 2)


def test_host_entry_matches_device_entry(bfm):
    """bfm_monitor_host (host buffers, chunked H2D/compute/D2H overlap) gives
    bit-identical outputs to bfm_monitor on device buffers."""
    w = synth.workload("c1", m=3000)
    dev = _run(bfm, w, w["Y"])
    d = bfm.Design(w["dates"], 3, 23.0)
    Yh = torch.from_numpy(w["Y"]).pin_memory()
    chunk = 512
    ws_bytes = bfm.bfm_monitor_host_workspace(d, 0, chunk, False)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    out = {k: torch.empty_like(torch.from_numpy(v)).pin_memory() for k, v in dev.items()}
    s = torch.cuda.current_stream()
    bfm.bfm_monitor_host(d, Yh, 0, None, 3000, w["n_hist"], w["h_frac"], w["lam"], out["break_idx"],
                         out["mean_mosum"], out["sigma"], out["beta"], out["status"], ws, ws_bytes, chunk, s)
    s.synchronize()
    for key in dev:
        np.testing.assert_array_equal(out[key].numpy(), dev[key])


@pytest.mark.parametrize("name,with_mask", [("c1", False), ("c3", False), ("c1", True)],
                         ids=["float", "int16", "float-mask"])
def test_host_entry_matches_oracle(bfm, name, with_mask):
    """bfm_monitor_host from pinned host buffers (Y float or int16, optional
    host mask bits) against the FP64 oracle element by element.  The chunk of
    384 pixels holds one and a half 256-pixel kernel tiles, so chunk and tile
    boundaries differ, and 3000 pixels leave a ragged last chunk of 312."""
    m, chunk = 3000, 384
    w = synth.workload(name, m=m)
    Y = np.ascontiguousarray(w["Y"])
    dtype = 1 if Y.dtype == np.int16 else 0
    mask = None
    if with_mask:
        rng = np.random.default_rng(5)
        mask = rng.integers(0, 2**32, size=(w["N"], (m + 31) // 32), dtype=np.uint64).astype(np.uint32)
        mask |= rng.integers(0, 2**32, size=mask.shape, dtype=np.uint64).astype(np.uint32)   # ~75 % set
    d = bfm.Design(w["dates"], w["k"], w["f"])
    K = d.K
    Yh = torch.from_numpy(Y).pin_memory()
    mh = None if mask is None else torch.from_numpy(mask.view(np.int32)).pin_memory()
    ws_bytes = bfm.bfm_monitor_host_workspace(d, dtype, chunk, with_mask)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    out = dict(break_idx=torch.empty(m, dtype=torch.int32).pin_memory(),
               mean_mosum=torch.empty(m, dtype=torch.float32).pin_memory(),
               sigma=torch.empty(m, dtype=torch.float32).pin_memory(),
               beta=torch.empty((K, m), dtype=torch.float32).pin_memory(),
               status=torch.empty(m, dtype=torch.uint8).pin_memory())
    s = torch.cuda.current_stream()
    bfm.bfm_monitor_host(d, Yh, dtype, mh, m, w["n_hist"], w["h_frac"], w["lam"], out["break_idx"],
                         out["mean_mosum"], out["sigma"], out["beta"], out["status"], ws, ws_bytes, chunk, s)
    s.synchronize()
    assert bfm.bfm_device_errors() == 0
    gpu = {k: v.numpy() for k, v in out.items()}
    rep, ref = _check(w, Y, gpu, mask=mask)
    assert (ref["break_idx"] >= 0).sum() > 300


def test_invalid_arguments(bfm):
    w = synth.workload("c1", m=64)
    d = bfm.Design(w["dates"], 3, 23.0)
    Yd = torch.from_numpy(w["Y"]).cuda()
    o = bfm.empty_outputs(8, 64)
    for kw in (dict(n_hist=0), dict(n_hist=w["N"]), dict(h_frac=0.0), dict(h_frac=1.5), dict(lam=-1.0)):
        args = dict(n_hist=w["n_hist"], h_frac=0.25, lam=1.7)
        args.update(kw)
        with pytest.raises(bfm.BfmError) as ei:
            bfm.monitor(d, Yd, out=o, **args)
        assert ei.value.code == 1
    with pytest.raises(bfm.BfmError):
        bfm.Design(w["dates"][::-1].copy(), 3, 23.0)
    with pytest.raises(bfm.BfmError):
        bfm.Design(w["dates"], 4, 23.0)


@pytest.fixture(scope="module")
def c2_full(bfm):
    """The full c2 scene (8,388,608 px x 414 dates, 13.9 GB float32) on the
    device, run once per form in the benchmark's launch configuration."""
    w = synth.workload("c2")
    Yd = torch.from_numpy(w["Y"]).cuda()
    d = bfm.Design(w["dates"], 3, 23.0)
    res = {}
    for algo in (1, 2, 4, 5):
        out = bfm.monitor(d, Yd, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"], algo=algo)
        torch.cuda.synchronize()
        assert bfm.bfm_device_errors() == 0
        res[algo] = to_numpy(out)
        if algo == 2:
            # bfm_trace of sampled pixels while the scene is resident (offsets t*m + p beyond 2^31)
            rng = np.random.default_rng(5)
            brk = np.nonzero(res[2]["break_idx"] >= 0)[0]
            sel = np.unique(np.concatenate([[0, w["m"] - 1], rng.choice(brk, 256, replace=False),
                                            rng.choice(w["m"], 256, replace=False)])).astype(np.int64)
            tr = bfm.trace(d, Yd, n_hist=w["n_hist"], h_frac=w["h_frac"], status=out["status"],
                           pixels=torch.from_numpy(sel).cuda())
            torch.cuda.synchronize()
            res["trace"] = (sel, tr["mo"].cpu().numpy(), tr["resid"].cpu().numpy())
        del out
    del Yd
    torch.cuda.empty_cache()
    return w, res


@ALGOS
def test_c2_full_scene_sampled(c2_full, algo):
    """Full-size scene; the oracle checks a seeded sample of 4096 pixels
    (including the first and last tiles) one by one."""
    w, res = c2_full
    res = res[algo]
    m = w["m"]
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([np.arange(64), np.arange(m - 64, m), rng.choice(m, 3968, replace=False)]))
    Ys = np.ascontiguousarray(w["Y"][:, idx])
    gpu = {k: (v[:, idx] if v.ndim == 2 else v[idx]) for k, v in res.items()}
    ws = dict(w, m=idx.size)
    _check(ws, Ys, gpu)


def test_c2_full_scene_trace(c2_full):
    """bfm_trace on the full-size scene: residuals and MO process of 514
    sampled pixels (half of them with a break) against the oracle run on
    those pixels' columns."""
    w, res = c2_full
    sel, mo, rs = res["trace"]
    Ys = np.ascontiguousarray(w["Y"][:, sel])
    ref = oracle.monitor(w["dates"], Ys, k=3, f=23.0, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"],
                         trace=True)
    ref["n_hist"] = w["n_hist"]
    vals, valid = oracle.valid_and_values(Ys)
    X = oracle.design(w["dates"], 3, 23.0)
    wm, wr, nb = check_trace_rows(np.arange(sel.size), mo, rs, ref, vals, valid, X, w["lam"], m=sel.size)
    print("worst MO error", wm, "worst residual error / max|y|", wr, "breaks checked", nb)
    assert nb > 100


@ALGOS
def test_c2_full_scene_properties(c2_full, algo):
    """Properties that hold at any size: every pixel has a status, breaks
    lie in the monitoring period, detection of the injected shifts."""
    w, res = c2_full
    res = res[algo]
    st = res["status"]
    assert np.isin(st, [0, 1, 2, 3, 4]).all()
    b = res["break_idx"]
    assert ((b == -1) | ((b >= w["n_hist"]) & (b < w["N"]))).all()
    tb = w["true_break"]
    det = (b >= 0)
    assert det[tb >= 0].mean() > 0.8


@pytest.mark.parametrize("dtype", ["f32", "i16"])
@ALGOS
def test_max_mosum(bfm, algo, dtype):
    """bfm_monitor_ext's map of the largest-magnitude MO (Section 4.3) against
    the oracle's MO trace: magnitudes within the form's tolerance, the sign
    wherever the runner-up magnitude is not within 1e-4 of the largest (the
    first of near-equal values may differ by rounding)."""
    w = synth.workload("c1" if dtype == "f32" else "c3", m=1024)
    d = bfm.Design(w["dates"], 3, 23.0)
    Yd = torch.from_numpy(w["Y"]).cuda()
    out = bfm.monitor(d, Yd, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"], algo=algo, max_mosum=True)
    torch.cuda.synchronize()
    assert bfm.bfm_device_errors() == 0
    g = out["max_mosum"].cpu().numpy().astype(np.float64)
    ref = oracle.monitor(w["dates"], w["Y"], k=3, f=23.0, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"],
                         trace=True)
    r = oracle.max_mosum(ref)
    st = out["status"].cpu().numpy()
    assert (st == ref["status"]).all()
    assert (np.isnan(g) == np.isnan(r)).all()
    ok = ~np.isnan(r)
    tol = 1e-5 if dtype == "f32" else 1e-4
    err = np.abs(np.abs(g[ok]) - np.abs(r[ok])) / np.maximum(1.0, np.abs(r[ok]))
    print("max |max_mosum| error", err.max())
    assert err.max() < tol
    tr = np.abs(np.nan_to_num(ref["mo_trace"], nan=0.0))
    srt = np.sort(tr, axis=1)
    clear = ok & (srt[:, -1] - srt[:, -2] > 1e-4 * np.maximum(1.0, srt[:, -1]))
    assert (np.sign(g[clear]) == np.sign(r[clear])).all()
