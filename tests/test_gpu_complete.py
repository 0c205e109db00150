"""The complete-series form (BFM_ALGO_COMPLETE: one shared pseudo-inverse,
Section 3, Eq. 8-11) against the FP64 oracle, element by element, through the
C ABI; and against the general forms on the same data.

Tolerances as for the float path (1e-5: beta column-scaled, sigma relative,
mean MOSUM relative to max(1, |ref|)); break indices equal except on
margin-tied pixels.
"""
import numpy as np
import pytest

import oracle
import synth
from _parity import compare, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def bfm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_01751_gb300 as bfm
    bfm.load()
    return bfm


def complete_scene(m, dtype="f32", N=228, n_hist=100, seed=21, date_vals=None):
    """The c1 recipe (K = 8 fit of a 2-harmonic signal, 20 % steps of -0.3)
    without missing values."""
    d, Y, brk = synth.scene(seed=seed, m=m, N=N, n_hist=n_hist, f=23.0, k_gen=2, intercept=0.5, slope=0.001,
                            coef_fixed=[0.2, 0.0, 0.0, 0.05], noise_sd=0.03, miss="none", break_frac=0.2,
                            step=(-0.3, -0.3), dtype=dtype, date_vals=date_vals)
    return dict(dates=d, Y=Y, true_break=brk, m=m, N=N, n_hist=n_hist, f=23.0, k=3, h_frac=0.25,
                lam=synth.workload_lambda("c1"))


def run(bfm, w, Y, *, k=3, algo=3, mask=None, max_mosum=False):
    d = bfm.Design(w["dates"], k, w["f"])
    Yd = torch.from_numpy(np.ascontiguousarray(Y)).cuda()
    md = None if mask is None else torch.from_numpy(mask.view(np.int32)).cuda()
    out = bfm.monitor(d, Yd, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"], mask_bits=md, algo=algo,
                      max_mosum=max_mosum)
    torch.cuda.synchronize()
    assert bfm.bfm_device_errors() == 0
    return to_numpy(out)


def oracle_of(w, Y, *, k=3, mask=None, trace=False):
    return oracle.monitor(w["dates"], Y, k=k, f=w["f"], n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"],
                          mask_bits=mask, trace=trace)


@pytest.mark.parametrize("dtype", ["f32", "i16"])
def test_complete_matches_oracle(bfm, dtype):
    """4136 pixels (16 full 256-pixel tiles and a ragged one; a multiple of 8
    so that the tensor-core form takes the same array)."""
    w = complete_scene(4136, dtype)
    gpu = run(bfm, w, w["Y"])
    ref = oracle_of(w, w["Y"])
    rep = compare(gpu, ref, w["dates"], 3, w["f"], tol=TOL)
    print(rep)
    assert rep["ok"], rep
    assert (ref["break_idx"] >= 0).sum() > 500
    # the general forms on the same data: same statuses, same breaks away from ties
    for algo in (1, 2):
        other = run(bfm, w, w["Y"], algo=algo)
        assert (other["status"] == gpu["status"]).all()
        untied = ref["margin"] >= 1e-5
        assert (other["break_idx"][untied] == gpu["break_idx"][untied]).all()


@pytest.mark.parametrize("k", [1, 2])
def test_complete_fewer_harmonics(bfm, k):
    w = complete_scene(1000)
    gpu = run(bfm, w, w["Y"], k=k)
    rep = compare(gpu, oracle_of(w, w["Y"], k=k), w["dates"], k, w["f"], tol=TOL)
    print(rep)
    assert rep["ok"], rep


@pytest.mark.parametrize("dtype,m", [("f32", 1001), ("i16", 1004)])
def test_complete_unaligned_rows(bfm, dtype, m):
    """Rows of Y that are not a multiple of 16 bytes cannot be bulk-copied:
    the plain-load form (register batches, the leaving residual recomputed)
    runs instead, with the same results."""
    w = complete_scene(m, dtype)
    gpu = run(bfm, w, w["Y"])
    rep = compare(gpu, oracle_of(w, w["Y"]), w["dates"], 3, w["f"], tol=TOL)
    print(rep)
    assert rep["ok"], rep


def test_complete_long_series(bfm):
    """The longest design (N = 1792, n_hist = 1200, h = 300): the shared
    table takes more than 48 KB of shared memory, the residual ring does not
    fit (plain-load form) and the history does not fit the L2 budget at two
    CTAs per SM."""
    w = complete_scene(700, N=1792, n_hist=1200)
    w["lam"] = synth.lambda_for_horizon(1792 / 1200)
    gpu = run(bfm, w, w["Y"])
    ref = oracle_of(w, w["Y"])
    # mean MOSUM: each of the h residuals of a window carries the FP32
    # rounding of its fitted value, up to 2^-24 max|y|, so the bound on a
    # window of h = 300 terms in MO units is h 2^-24 max|y| / (sigma sqrt(n))
    # (1.4e-5 .. 4e-5 here); beta and sigma keep 1e-5
    h = int(np.floor(w["h_frac"] * w["n_hist"]))
    ymax = np.abs(w["Y"][: w["n_hist"]]).max(axis=0)
    bound = np.maximum(TOL, h * 2.0 ** -24 * ymax / (ref["sigma"] * np.sqrt(w["n_hist"])))
    rep = compare(gpu, ref, w["dates"], 3, w["f"], tol=1.0)
    print(rep)
    assert rep["status_mismatch"] == 0 and rep["break_mismatch_untied"] == 0
    assert rep["beta_err_max"] <= TOL and rep["sigma_err_max"] <= TOL
    ok = ref["status"] == 0
    me = np.abs(gpu["mean_mosum"][ok] - ref["mean_mosum"][ok]) / np.maximum(1.0, np.abs(ref["mean_mosum"][ok]))
    print("mean MOSUM error / bound, max", (me / bound[ok]).max())
    assert (me <= bound[ok]).all()


def test_complete_incomplete_pixels(bfm):
    """Pixels with a missing value (NaN in the history or the monitoring
    period, a 0 mask bit) get INCOMPLETE and NaN outputs; the others are
    unaffected."""
    w = complete_scene(600)
    Y = w["Y"].copy()
    Y[5, 3] = np.nan
    Y[w["n_hist"] + 7, 10] = np.nan
    Y[w["N"] - 1, 599] = np.nan
    words = (600 + 31) // 32
    mask = np.full((w["N"], words), 0xFFFFFFFF, np.uint32)
    mask[50, 20 // 32] &= ~np.uint32(1 << (20 % 32))
    gpu = run(bfm, w, Y, mask=mask)
    bad = [3, 10, 599, 20]
    assert (gpu["status"][bad] == 5).all()
    assert (gpu["break_idx"][bad] == -1).all()
    assert np.isnan(gpu["mean_mosum"][bad]).all() and np.isnan(gpu["sigma"][bad]).all()
    assert np.isnan(gpu["beta"][:, bad]).all()
    good = np.setdiff1d(np.arange(600), bad)
    ref = oracle_of(w, Y, mask=mask)
    sub = lambda o: {kk: (v[:, good] if v.ndim == 2 else v[good]) for kk, v in o.items()}
    rep = compare(sub(gpu), sub(ref), w["dates"], 3, w["f"], tol=TOL)
    assert rep["ok"], rep
    # the same data without the mask and with the general form: those pixels are fitted there
    gen = run(bfm, w, Y, mask=mask, algo=2)
    assert (gen["status"][bad] != 5).all()


def test_complete_shared_status(bfm):
    """n_hist <= K gives INSUFFICIENT_HISTORY for every pixel; a singular
    shared design (whole-number dates with f = 1: every harmonic column is 0
    or equal to the intercept) gives SINGULAR for every pixel, as in the
    oracle."""
    w = complete_scene(300)
    w8 = dict(w, n_hist=8)
    gpu = run(bfm, w8, w["Y"])
    assert (gpu["status"] == 1).all() and np.isnan(gpu["sigma"]).all() and (gpu["break_idx"] == -1).all()
    assert (oracle_of(w8, w["Y"])["status"] == 1).all()
    ws = complete_scene(300, date_vals=np.arange(228, dtype=np.float64))
    ws["f"] = 1.0
    gpu = run(bfm, ws, ws["Y"])
    ref = oracle_of(ws, ws["Y"])
    assert (ref["status"] == 2).all()
    assert (gpu["status"] == 2).all() and np.isnan(gpu["beta"]).all()


def test_complete_degenerate(bfm):
    """Constant and noise-free harmonic series: sigma-hat at rounding level,
    DEGENERATE (MO = 0, mean 0, no break), as in the oracle."""
    w = complete_scene(256)
    Y = w["Y"].copy()
    Y[:, 0] = 0.25
    t = w["dates"]
    Y[:, 1] = (0.5 + 0.2 * np.sin(2 * np.pi * t / 23.0)).astype(np.float32)
    gpu = run(bfm, w, Y, max_mosum=True)
    ref = oracle_of(w, Y)
    assert list(gpu["status"][:2]) == [3, 3] and list(ref["status"][:2]) == [3, 3]
    assert (gpu["mean_mosum"][:2] == 0).all() and (gpu["break_idx"][:2] == -1).all()
    assert (gpu["max_mosum"][:2] == 0).all()
    rep = compare(gpu, ref, w["dates"], 3, w["f"], tol=TOL)
    assert rep["ok"], rep


@pytest.mark.parametrize("dtype", ["f32", "i16"])
def test_complete_max_mosum(bfm, dtype):
    w = complete_scene(1024, dtype)
    gpu = run(bfm, w, w["Y"], max_mosum=True)
    ref = oracle_of(w, w["Y"], trace=True)
    r = oracle.max_mosum(ref)
    g = gpu["max_mosum"].astype(np.float64)
    assert (np.isnan(g) == np.isnan(r)).all()
    ok = ~np.isnan(r)
    err = np.abs(np.abs(g[ok]) - np.abs(r[ok])) / np.maximum(1.0, np.abs(r[ok]))
    print("max |max_mosum| error", err.max())
    assert err.max() < TOL
    tr = np.abs(np.nan_to_num(ref["mo_trace"], nan=0.0))
    srt = np.sort(tr, axis=1)
    clear = ok & (srt[:, -1] - srt[:, -2] > 1e-4 * np.maximum(1.0, srt[:, -1]))
    assert (np.sign(g[clear]) == np.sign(r[clear])).all()


def test_complete_full_scene_sampled(bfm):
    """The cloud-free c2 scene at full size (8,388,608 px x 414 dates, device
    generated) in the benchmark's launch configuration; the oracle checks a
    seeded sample of 4096 pixels (first and last tiles included) one by one,
    and the tensor-core form on the same scene agrees on statuses and on
    untied breaks."""
    w = synth.workload_torch("c2_complete", device="cuda")
    m = w["m"]
    d = bfm.Design(w["dates"], 3, 23.0)
    out = bfm.monitor(d, w["Y"], n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"], algo=3)
    gen = bfm.monitor(d, w["Y"], n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"], algo=2)
    torch.cuda.synchronize()
    assert bfm.bfm_device_errors() == 0
    rng = np.random.default_rng(3)
    idx = np.unique(np.concatenate([np.arange(64), np.arange(m - 64, m), rng.choice(m, 3968, replace=False)]))
    it = torch.from_numpy(idx).cuda()
    Ys = w["Y"].index_select(1, it).cpu().numpy()
    gpu = {k: (v.index_select(1, it) if v.dim() == 2 else v.index_select(0, it)).cpu().numpy()
           for k, v in out.items()}
    ref = oracle.monitor(w["dates"], Ys, k=3, f=23.0, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"])
    rep = compare(gpu, ref, w["dates"], 3, 23.0, tol=TOL)
    print(rep)
    assert rep["ok"], rep
    st = out["status"].cpu().numpy()
    assert (st == gen["status"].cpu().numpy()).all()
    assert (st == 0).mean() > 0.99
    b1, b2 = out["break_idx"].cpu().numpy(), gen["break_idx"].cpu().numpy()
    print("break mismatches between the forms over the scene", int((b1 != b2).sum()))
    assert (b1 != b2).mean() < 1e-4
