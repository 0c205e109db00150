"""bfm_trace (residuals and MOSUM process of selected pixels, Section 3.2)
against the FP64 oracle, through the C ABI.

The oracle's MO trace lists MO_j by monitoring position; here it is mapped to
the original dates of the pixel's valid observations.  Reference residuals are
y - x'beta at the valid dates with the oracle's beta (Householder QR, raw
Eq. 2 design).  Both sides are FP64 up to the float output, so the tolerance
is the float rounding of the output plus 1e-9 relative.
"""
import numpy as np
import pytest

import oracle
import synth
from _parity import check_trace_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bfm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_01751_gb300 as bfm
    bfm.load()
    return bfm


def _bits(N, m, seed):
    rng = np.random.default_rng(seed)
    words = (m + 31) // 32
    keep = rng.random((N, words * 32)) > 0.2
    bits = np.zeros((N, words), np.uint32)
    for b in range(32):
        bits |= keep[:, b::32].astype(np.uint32) << np.uint32(b)
    return bits


@pytest.mark.parametrize("masked", [False, True], ids=["nan", "mask_bits"])
@pytest.mark.parametrize("dtype", ["f32", "i16"])
def test_trace_matches_oracle(bfm, dtype, masked):
    w = synth.workload("c1" if dtype == "f32" else "c3", m=1024)
    Y = w["Y"]
    N, m = Y.shape
    bits = _bits(N, m, 11) if masked else None
    d = bfm.Design(w["dates"], 3, 23.0)
    Yd = torch.from_numpy(Y).cuda()
    md = None if bits is None else torch.from_numpy(bits.view(np.int32)).cuda()
    out = bfm.monitor(d, Yd, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"], mask_bits=md)
    ref = oracle.monitor(w["dates"], Y, k=3, f=23.0, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"],
                         mask_bits=bits, trace=True)
    ref["n_hist"] = w["n_hist"]
    st = out["status"].cpu().numpy()
    assert (st == ref["status"]).all()
    brk = np.nonzero(ref["break_idx"] >= 0)[0]
    quiet = np.nonzero(ref["break_idx"] < 0)[0]
    other = np.nonzero(st != 0)[0]
    sel = np.concatenate([brk[:300], quiet[:150], other[:40], [m + 5, -1, 0, m - 1]]).astype(np.int64)
    pix = torch.from_numpy(sel).cuda()
    tr = bfm.trace(d, Yd, n_hist=w["n_hist"], h_frac=w["h_frac"], status=out["status"], pixels=pix, mask_bits=md)
    torch.cuda.synchronize()
    assert bfm.bfm_device_errors() == 0
    vals, valid = oracle.valid_and_values(Y, bits)
    X = oracle.design(w["dates"], 3, 23.0)
    wm, wr, nb = check_trace_rows(sel, tr["mo"].cpu().numpy(), tr["resid"].cpu().numpy(), ref, vals, valid, X,
                                  w["lam"], m=m)
    print("worst MO error", wm, "worst residual error / max|y|", wr, "breaks checked", nb)
    assert nb > 100


def test_trace_first_pixels_mo_only(bfm):
    """pixels = NULL (the first `count` pixels) and resid = NULL."""
    w = synth.workload("c1", m=256)
    d = bfm.Design(w["dates"], 3, 23.0)
    Yd = torch.from_numpy(w["Y"]).cuda()
    out = bfm.monitor(d, Yd, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"])
    tr = bfm.trace(d, Yd, n_hist=w["n_hist"], h_frac=w["h_frac"], status=out["status"], count=200, resid=False)
    torch.cuda.synchronize()
    assert "resid" not in tr and tr["mo"].shape == (200, w["N"])
    ref = oracle.monitor(w["dates"], w["Y"], k=3, f=23.0, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"],
                         trace=True)
    ref["n_hist"] = w["n_hist"]
    vals, valid = oracle.valid_and_values(w["Y"])
    X = oracle.design(w["dates"], 3, 23.0)
    check_trace_rows(np.arange(200), tr["mo"].cpu().numpy(), None, ref, vals, valid, X, w["lam"], m=256)


@pytest.mark.parametrize("k", [1, 2])
def test_trace_fewer_harmonics(bfm, k):
    w = synth.workload("c1", m=512)
    d = bfm.Design(w["dates"], k, 23.0)
    Yd = torch.from_numpy(w["Y"]).cuda()
    out = bfm.monitor(d, Yd, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"])
    tr = bfm.trace(d, Yd, n_hist=w["n_hist"], h_frac=w["h_frac"], status=out["status"], count=512)
    torch.cuda.synchronize()
    ref = oracle.monitor(w["dates"], w["Y"], k=k, f=23.0, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"],
                         trace=True)
    ref["n_hist"] = w["n_hist"]
    assert (out["status"].cpu().numpy() == ref["status"]).all()
    vals, valid = oracle.valid_and_values(w["Y"])
    X = oracle.design(w["dates"], k, 23.0)
    check_trace_rows(np.arange(512), tr["mo"].cpu().numpy(), tr["resid"].cpu().numpy(), ref, vals, valid, X,
                     w["lam"], m=512)


def test_trace_degenerate_and_short(bfm):
    """Constant series (DEGENERATE: MO = 0), almost empty series
    (INSUFFICIENT_HISTORY: NaN rows), series without monitoring data."""
    w = synth.workload("c1", m=128)
    Y = w["Y"].copy()
    Y[:, 0] = 0.25                       # constant: sigma-hat = 0
    Y[:, 1] = np.nan
    Y[:5, 1] = 0.3                       # 5 observations: no fit
    Y[w["n_hist"]:, 2] = np.nan          # nothing to monitor
    d = bfm.Design(w["dates"], 3, 23.0)
    Yd = torch.from_numpy(Y).cuda()
    out = bfm.monitor(d, Yd, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"])
    st = out["status"].cpu().numpy()
    assert list(st[:3]) == [3, 1, 4]
    tr = bfm.trace(d, Yd, n_hist=w["n_hist"], h_frac=w["h_frac"], status=out["status"], count=128)
    torch.cuda.synchronize()
    ref = oracle.monitor(w["dates"], Y, k=3, f=23.0, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"],
                         trace=True)
    ref["n_hist"] = w["n_hist"]
    vals, valid = oracle.valid_and_values(Y)
    X = oracle.design(w["dates"], 3, 23.0)
    mo = tr["mo"].cpu().numpy()
    rs = tr["resid"].cpu().numpy()
    assert (mo[0, w["n_hist"]:] == 0).all() and np.isnan(mo[0, : w["n_hist"]]).all()
    assert np.abs(rs[0]).max() < 1e-6
    check_trace_rows(np.arange(128), mo, rs, ref, vals, valid, X, w["lam"], m=128)


def test_trace_arguments(bfm):
    w = synth.workload("c1", m=64)
    d = bfm.Design(w["dates"], 3, 23.0)
    Yd = torch.from_numpy(w["Y"]).cuda()
    st = torch.zeros(64, dtype=torch.uint8, device="cuda")
    mo = torch.empty((4, w["N"]), device="cuda")
    # count = 0 enqueues nothing, even without outputs
    bfm.bfm_trace(d, Yd, 0, None, 64, w["n_hist"], 0.25, None, 0, st, None, None)
    for args in ((64, w["n_hist"], 0.25, 4, st, None, None),     # no output
                 (64, w["N"], 0.25, 4, st, mo, None),             # n_hist >= N
                 (64, w["n_hist"], 0.0, 4, st, mo, None),         # h_frac
                 (64, w["n_hist"], 0.25, 4, None, mo, None),      # no status
                 (0, w["n_hist"], 0.25, 4, st, mo, None)):        # m = 0
        m, nh, hf, cnt, s, o, r = args
        with pytest.raises(bfm.BfmError) as ei:
            bfm.bfm_trace(d, Yd, 0, None, m, nh, hf, None, cnt, s, o, r)
        assert ei.value.code == 1
