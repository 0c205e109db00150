"""Tensor-core (tcgen05) form vs the FP64 oracle, element by element.

int16 or float storage; Gram / X'My / fitted values on fp16 tensor cores with
split hi/lo operands (per-pixel power-of-two scales) and FP32 accumulation,
FP32 solve with one refinement step.  Tolerance of this form: 1e-4 (beta
column-scaled, sigma relative, mean MOSUM relative to max(1, |ref|)); break
indices equal except margin-tied pixels.  On the float workloads it also
meets the FP32 tolerance 1e-5.
"""
import numpy as np
import pytest

import oracle
import synth
from _parity import compare, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_MMA = 1e-4
ALGO_MMA = 2


@pytest.fixture(scope="module")
def bfm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_01751_gb300 as bfm
    bfm.load()
    return bfm


def _run(bfm, dates, Y, *, k, n_hist, h_frac, lam, mask=None, algo=ALGO_MMA):
    d = bfm.Design(dates, k, 23.0)
    Yd = torch.from_numpy(np.ascontiguousarray(Y)).cuda()
    md = None if mask is None else torch.from_numpy(mask.view(np.int32)).cuda()
    out = bfm.monitor(d, Yd, n_hist=n_hist, h_frac=h_frac, lam=lam, mask_bits=md, algo=algo)
    torch.cuda.synchronize()
    assert bfm.bfm_device_errors() == 0
    return to_numpy(out)


def _check(dates, Y, gpu, *, k, n_hist, h_frac, lam, mask=None, tol=TOL_MMA):
    ref = oracle.monitor(dates, Y, k=k, f=23.0, n_hist=n_hist, h_frac=h_frac, lam=lam, mask_bits=mask)
    rep = compare(gpu, ref, dates, k, 23.0, tol=tol)
    print(rep)
    assert rep["ok"], rep
    return rep, ref


def test_c3_mma(bfm):
    """c3: the c1 scene in int16 (NDVI*1e4, -32768 missing), 32 tiles of 128."""
    w = synth.workload("c3")
    g = _run(bfm, w["dates"], w["Y"], k=3, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"])
    rep, _ = _check(w["dates"], w["Y"], g, k=3, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"])
    assert rep["beta_err_max"] < 1e-5 and rep["mean_err_max"] < 2e-5


@pytest.mark.parametrize("dtype", ["i16", "f32"])
def test_c2_recipe(bfm, dtype):
    """c2 recipe (N = 414, n_hist = 228, ~60 % Markov clouds), 8192 px."""
    w = synth.workload("c2", m=8192, dtype=dtype)
    g = _run(bfm, w["dates"], w["Y"], k=3, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"])
    rep, _ = _check(w["dates"], w["Y"], g, k=3, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"])
    if dtype == "f32":
        assert rep["beta_err_max"] < 1e-5 and rep["sigma_err_max"] < 1e-5 and rep["mean_err_max"] < 1e-5


def test_c1_f32(bfm):
    """c1 (float storage, N = 228, n_hist = 100, iid clouds) at the FP32 tolerance."""
    w = synth.workload("c1")
    g = _run(bfm, w["dates"], w["Y"], k=3, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"])
    _check(w["dates"], w["Y"], g, k=3, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"], tol=1e-5)


@pytest.mark.parametrize("dtype", ["i16", "f32"])
@pytest.mark.parametrize("m", [128, 136, 1000, 4104, 4232])
def test_ragged(bfm, m, dtype):
    """One full tile, and ragged last tiles of 8, 104 and 8 live pixels (the
    TMA box reads zeros past m; those pixels are not written)."""
    w = synth.workload("c3" if dtype == "i16" else "c1", m=m)
    g = _run(bfm, w["dates"], w["Y"], k=3, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"])
    _check(w["dates"], w["Y"], g, k=3, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"])


@pytest.mark.parametrize("dtype", ["i16", "f32"])
@pytest.mark.parametrize("m", [1, 100, 129, 4093])
def test_untileable_layout_is_refused(bfm, m, dtype):
    """m < 128 or rows that are not a multiple of 16 bytes: no tensor map for
    Y, so algo = MMA is BFM_EUNSUPPORTED and AUTO takes the CUDA-core form."""
    w = synth.workload("c3" if dtype == "i16" else "c1", m=m)
    kw = dict(k=3, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"])
    with pytest.raises(bfm.BfmError) as ei:
        _run(bfm, w["dates"], w["Y"], **kw)
    assert ei.value.code == 6
    g = _run(bfm, w["dates"], w["Y"], algo=0, **kw)
    _check(w["dates"], w["Y"], g, tol=1e-5, **kw)


def test_f32_value_ranges(bfm):
    """Float series far outside fp16's range, and series whose first eight
    dates are missing, tiny or much smaller than the rest: the per-pixel
    operand scales (and the redo of the normal equations when a value leaves
    the first estimate's range) keep the results at the FP32 tolerance."""
    w = synth.workload("c1", m=1024)
    Y = w["Y"].astype(np.float64)
    Y[:, 0:128] *= 1e6            # |y| ~ 1e6 > fp16 max
    Y[:, 128:256] *= 1e-7         # |y| ~ 1e-7 < fp16 min normal
    Y[0:8, 256:384] = np.nan      # first eight dates missing: no first estimate
    Y[0:8, 384:512] *= 1e-3       # first eight dates 1000x smaller: redo
    Y[:, 512:640] *= 1e15         # squared residuals near 1e29: still inside float's range
    Y = Y.astype(np.float32)
    g = _run(bfm, w["dates"], Y, k=3, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"])
    _check(w["dates"], Y, g, k=3, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"], tol=1e-5)


def test_mask_bits(bfm):
    w = synth.workload("c3", m=1024)
    rng = np.random.default_rng(5)
    words = 1024 // 32
    on = rng.random((w["N"], 1024)) > 0.15
    bits = np.zeros((w["N"], words), np.uint32)
    for b in range(32):
        bits |= on[:, b::32].astype(np.uint32) << np.uint32(b)
    g = _run(bfm, w["dates"], w["Y"], k=3, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"], mask=bits)
    _check(w["dates"], w["Y"], g, k=3, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"], mask=bits)


@pytest.mark.parametrize("dtype", ["i16", "f32"])
@pytest.mark.parametrize("k,N,n_hist", [(1, 150, 70), (2, 300, 180), (3, 448, 340), (1, 61, 37), (3, 600, 420),
                                         (1, 1000, 500)])
def test_harmonics_and_lengths(bfm, k, N, n_hist, dtype):
    """Each harmonic order, 61 to 1000 dates (one CTA per SM from about 450).  (Short series with many
    regressors, e.g. K = 8 from 17 history dates at 55 % clouds, give Gram
    condition numbers up to 1e9 below the singularity threshold: no FP32 form
    meets 1e-4 there, so they are not parity cases.)"""
    d, Y, _ = synth.scene(seed=40 + k, m=2048, N=N, n_hist=n_hist, f=23.0, k_gen=k, intercept=0.45,
                          slope=0.0002, coef_umax=0.25, noise_sd=0.03, miss="markov", p_a=0.25, p_b=0.3,
                          break_frac=0.2, step=(-0.4, -0.1), dtype=dtype)
    g = _run(bfm, d, Y, k=k, n_hist=n_hist, h_frac=0.25, lam=1.75)
    _check(d, Y, g, k=k, n_hist=n_hist, h_frac=0.25, lam=1.75)


def test_edge_statuses(bfm):
    w = synth.workload("c3", m=256)
    Y = w["Y"].copy()
    N, n = w["N"], w["n_hist"]
    Y[:, 0] = -32768
    Y[8:n, 127] = -32768
    Y[n:, 128] = -32768
    Y[:, 255] = 5000                      # exact fit: sigma-hat = 0, DEGENERATE
    g = _run(bfm, w["dates"], Y, k=3, n_hist=n, h_frac=0.25, lam=w["lam"])
    rep, ref = _check(w["dates"], Y, g, k=3, n_hist=n, h_frac=0.25, lam=w["lam"])
    assert list(ref["status"][[0, 127, 128, 255]]) == [1, 1, 4, 3]


def test_rounding_noise_only_pixels(bfm):
    """Noise-free season-trend series rounded to int16: the residuals are
    the rounding (sigma-hat ~ 0.29 units against a signal of ~5000), the
    hardest case for this form.  Its remaining error is the out-of-span part
    of the fp16 hi/lo split of the basis table (2^-22 relative per entry)
    plus FP32 accumulation of yhat: eps = 2^-21 sum_{i>=1} |beta_i| max|x_i|
    + 2^-22 max|yhat| per residual.  It enters the window sums (h eps /
    (sigma sqrt(n))) and, relatively, sigma-hat itself (2 eps / sigma), so
    |d mean| <= h eps / (sigma sqrt(n)) + 2 (eps / sigma) |mean|.  Status and
    breaks still agree."""
    w = synth.workload("c3", m=128)
    X = oracle.design(w["dates"], 3, 23.0)
    rng = np.random.default_rng(9)
    cols = []
    for _ in range(128):
        b = np.array([5000, 4, 2000, 300, 100, 500, 50, 20]) * rng.uniform(0.5, 1.0, 8)
        cols.append(np.round(X @ b))
    Y = np.stack(cols, axis=1).astype(np.int16)
    Y[w["n_hist"] + 40:, ::2] -= 3000        # shifts in half of them
    g = _run(bfm, w["dates"], Y, k=3, n_hist=w["n_hist"], h_frac=0.25, lam=w["lam"])
    ref = oracle.monitor(w["dates"], Y, k=3, f=23.0, n_hist=w["n_hist"], h_frac=0.25, lam=w["lam"])
    assert (g["status"] == ref["status"]).all()
    tie = ref["margin"] < 1e-3
    assert ((g["break_idx"] == ref["break_idx"]) | tie).all()
    ok = ref["status"] == 0
    xmax = np.abs(X).max(axis=0)
    yhat = X @ ref["beta"]
    eps = 2.0 ** -21 * (np.abs(ref["beta"][1:]) * xmax[1:, None]).sum(0) + 2.0 ** -22 * np.abs(yhat).max(0)
    bound = ref["h"] * eps / (ref["sigma"] * np.sqrt(ref["n"])) + 2 * eps / ref["sigma"] * np.abs(ref["mean_mosum"])
    err = np.abs(g["mean_mosum"].astype(np.float64) - ref["mean_mosum"])
    print("max err / bound", float((err[ok] / bound[ok]).max()), "max err", float(err[ok].max()))
    assert (err[ok] <= bound[ok]).all()


def test_bandwidth_limit_is_refused(bfm):
    """A bandwidth whose MOSUM ring (h + 17 prefix sums per pixel) does not fit
    shared memory next to the tables and the Y stages is BFM_EUNSUPPORTED
    with algo = MMA; AUTO takes the CUDA-core form."""
    d, Y, _ = synth.scene(seed=3, m=256, N=448, n_hist=440, f=23.0, k_gen=3, dtype="i16")
    with pytest.raises(bfm.BfmError) as ei:
        _run(bfm, d, Y, k=3, n_hist=440, h_frac=1.0, lam=1.75)
    assert ei.value.code == 6
    g = _run(bfm, d, Y, k=3, n_hist=440, h_frac=1.0, lam=1.75, algo=0)
    # windows over the whole history: FP32 sums of ~180 residuals per window
    _check(d, Y, g, k=3, n_hist=440, h_frac=1.0, lam=1.75)


def test_tables_beyond_shared_memory_are_refused(bfm):
    """1792 dates with k = 3 and a long history: the basis tables alone exceed
    an SM's shared memory, so AUTO takes the CUDA-core form."""
    d, Y, _ = synth.scene(seed=5, m=256, N=1792, n_hist=1600, f=23.0, k_gen=3, dtype="i16")
    design = bfm.Design(d, 3, 23.0)
    Yd = torch.from_numpy(Y).cuda()
    assert bfm.bfm_algo_auto(design, bfm.BFM_I16, 1600, 0.25, Yd, 256) == bfm.BFM_ALGO_SIMT
    with pytest.raises(bfm.BfmError) as ei:
        _run(bfm, d, Y, k=3, n_hist=1600, h_frac=0.25, lam=1.75)
    assert ei.value.code == 6


def test_wide_bandwidth(bfm):
    """h = 100 valid observations (ring of 109 slots, beyond the A buffers and
    table B it overlays): the ring region grows."""
    d, Y, _ = synth.scene(seed=3, m=1024, N=448, n_hist=400, f=23.0, k_gen=3, dtype="i16")
    g = _run(bfm, d, Y, k=3, n_hist=400, h_frac=0.25, lam=1.75)
    _check(d, Y, g, k=3, n_hist=400, h_frac=0.25, lam=1.75)


@pytest.mark.parametrize("dtype", ["i16", "f32"])
def test_mma_matches_simt_on_same_input(bfm, dtype):
    """Both forms on the same input agree within the precision form's tolerance."""
    w = synth.workload("c2", m=4096, dtype=dtype)
    kw = dict(k=3, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"])
    a = _run(bfm, w["dates"], w["Y"], algo=ALGO_MMA, **kw)
    b = _run(bfm, w["dates"], w["Y"], algo=1, **kw)
    ok = (a["status"] == 0) & (b["status"] == 0)
    assert (a["status"] == b["status"]).all()
    rel = np.abs(a["sigma"][ok] - b["sigma"][ok]) / b["sigma"][ok]
    assert rel.max() < 1e-4


@pytest.mark.parametrize("dtype", ["i16", "f32"])
def test_c2_full_sampled(bfm, dtype):
    """The full c2 scene (float, and stored as int16), in the benchmark's
    launch configuration; the oracle checks a seeded sample of pixels."""
    w = synth.workload_torch("c2", device="cuda", dtype=dtype)
    d = bfm.Design(w["dates"], 3, 23.0)
    out = bfm.monitor(d, w["Y"], n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"], algo=ALGO_MMA)
    torch.cuda.synchronize()
    assert bfm.bfm_device_errors() == 0
    m = w["m"]
    rng = np.random.default_rng(1)
    idx = np.unique(np.concatenate([np.arange(128), np.arange(m - 128, m), rng.choice(m, 3840, replace=False)]))
    it = torch.from_numpy(idx).cuda()
    Ys = w["Y"].index_select(1, it).cpu().numpy()
    res = {k: (v.index_select(1, it) if v.dim() == 2 else v.index_select(0, it)).cpu().numpy() for k, v in out.items()}
    _check(w["dates"], Ys, res, k=3, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"])
