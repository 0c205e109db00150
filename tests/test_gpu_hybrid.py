"""The hybrid form (BFM_ALGO_HYBRID: tensor-core contractions, one thread per
pixel for the scans) against the FP64 oracle, element by element, through the
C ABI.

Tolerance 1e-5 (beta column-scaled, sigma relative, mean MOSUM relative to
max(1, |ref|)) for float and int16 storage; break indices equal except on
margin-tied pixels.  Cases: the c1 and c3 scenes, samples of the c2 recipe
(414 dates, 60 % Markov clouds) in float and int16, ragged pixel counts (a
last CTA tile with a few live pixels, fewer pixels than one M-tile), explicit
mask bits, k = 1..3, every pixel status on M-tile boundaries, the max |MO|
map, equality with the streaming CUDA-core form, and refusal of layouts the
form cannot take.
"""
import numpy as np
import pytest

import oracle
import synth
from _parity import compare, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HYBRID, STREAM = 5, 4
TOL = 1e-5


@pytest.fixture(scope="module")
def bfm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_01751_gb300 as bfm
    bfm.load()
    return bfm


def _run(bfm, w, Y, *, mask=None, k=None, algo=HYBRID, max_mosum=False):
    k = w["k"] if k is None else k
    d = bfm.Design(w["dates"], k, w["f"])
    Yd = torch.from_numpy(np.ascontiguousarray(Y)).cuda()
    md = None if mask is None else torch.from_numpy(mask.view(np.int32)).cuda()
    out = bfm.monitor(d, Yd, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"], mask_bits=md, algo=algo,
                      max_mosum=max_mosum)
    torch.cuda.synchronize()
    assert bfm.bfm_device_errors() == 0
    return to_numpy(out)


def _check(w, Y, gpu, *, k=None, mask=None, tol=TOL):
    k = w["k"] if k is None else k
    ref = oracle.monitor(w["dates"], Y, k=k, f=w["f"], n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"],
                         mask_bits=mask)
    rep = compare(gpu, ref, w["dates"], k, w["f"], tol=tol)
    print(rep)
    assert rep["ok"], rep
    return rep, ref


@pytest.mark.parametrize("name", ["c1", "c3"])
def test_c1_c3(bfm, name):
    w = synth.workload(name)
    gpu = _run(bfm, w, w["Y"])
    rep, ref = _check(w, w["Y"], gpu)
    assert (ref["break_idx"] >= 0).sum() > 500


@pytest.mark.parametrize("dtype", ["f32", "i16"])
def test_c2_recipe_sample(bfm, dtype):
    """The benchmark's recipe (N = 414, n_hist = 228, 60 % Markov clouds) on
    the first 24,576 pixels of the scene: 48 CTA tiles, several per CTA."""
    w = synth.workload("c2", m=24576, dtype=dtype)
    gpu = _run(bfm, w, w["Y"])
    rep, ref = _check(w, w["Y"], gpu)
    assert (ref["break_idx"] >= 0).sum() > 1000


@pytest.mark.parametrize("m,dtype", [(4100, "f32"), (4104, "i16"), (8, "f32"), (136, "i16")])
def test_ragged(bfm, m, dtype):
    """A last tile with a few live pixels (out-of-range box columns are
    zero-filled and never written), or fewer pixels than one M-tile."""
    w = synth.workload("c1" if dtype == "f32" else "c3", m=m)
    gpu = _run(bfm, w, w["Y"])
    _check(w, w["Y"], gpu)


def test_mask_bits(bfm):
    w = synth.workload("c1", m=1024)
    rng = np.random.default_rng(3)
    words = 1024 // 32
    mask = rng.random((w["N"], words * 32)) > 0.2
    bits = np.zeros((w["N"], words), np.uint32)
    for b in range(32):
        bits |= mask[:, b::32].astype(np.uint32) << np.uint32(b)
    gpu = _run(bfm, w, w["Y"], mask=bits)
    _check(w, w["Y"], gpu, mask=bits)


@pytest.mark.parametrize("k", [1, 2])
def test_fewer_harmonics(bfm, k):
    w = synth.workload("c1", m=2048)
    d, Y, _ = synth.scene(seed=21 + k, m=2048, N=w["N"], n_hist=w["n_hist"], f=23.0, k_gen=k, intercept=0.4,
                          slope=0.0005, coef_umax=0.2, noise_sd=0.02, miss="markov", p_a=0.3, p_b=0.3,
                          break_frac=0.2, step=(-0.4, -0.1))
    w2 = dict(w, dates=d)
    gpu = _run(bfm, w2, Y, k=k)
    _check(w2, Y, gpu, k=k)


def test_edge_statuses(bfm):
    """Pixels crafted for every status on M-tile and warp boundaries: all
    missing, too few history observations, no monitoring data, noise-free
    (degenerate), collinear history (singular)."""
    w = synth.workload("c1", m=1024)
    Y = w["Y"].copy()
    N, n = w["N"], w["n_hist"]
    Y[:, 0] = np.nan
    Y[8:n, 127] = np.nan
    Y[n:, 128] = np.nan
    X = oracle.design(w["dates"], 3, 23.0)
    Y[:, 511] = (X @ np.array([0.5, 0.001, 0.2, 0.0, 0.0, 0.05, 0.0, 0.0])).astype(np.float32)
    keep = np.zeros(N, bool)
    keep[np.arange(0, N, 23)] = True
    Y[~keep, 512] = np.nan
    gpu = _run(bfm, w, Y)
    rep, ref = _check(w, Y, gpu)
    assert ref["status"][0] == 1 and ref["status"][127] == 1 and ref["status"][128] == 4
    assert ref["status"][511] == 3 and ref["status"][512] in (1, 2)


@pytest.mark.parametrize("name", ["c1", "c3"])
def test_max_mosum(bfm, name):
    """The map of the largest-magnitude MO (Section 4.3) against the oracle's
    MO trace; the sign wherever the runner-up magnitude is not within 1e-4."""
    w = synth.workload(name, m=1024)
    out = _run(bfm, w, w["Y"], max_mosum=True)
    g = out["max_mosum"].astype(np.float64)
    ref = oracle.monitor(w["dates"], w["Y"], k=3, f=23.0, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"],
                         trace=True)
    r = oracle.max_mosum(ref)
    assert (out["status"] == ref["status"]).all()
    assert (np.isnan(g) == np.isnan(r)).all()
    ok = ~np.isnan(r)
    err = np.abs(np.abs(g[ok]) - np.abs(r[ok])) / np.maximum(1.0, np.abs(r[ok]))
    print("max |max_mosum| error", err.max())
    assert err.max() < TOL
    tr = np.abs(np.nan_to_num(ref["mo_trace"], nan=0.0))
    srt = np.sort(tr, axis=1)
    clear = ok & (srt[:, -1] - srt[:, -2] > 1e-4 * np.maximum(1.0, srt[:, -1]))
    assert (np.sign(g[clear]) == np.sign(r[clear])).all()


def test_matches_streaming_form(bfm):
    """Same statuses as the streaming CUDA-core form on the c2 recipe, and the
    same break wherever neither form is within 1e-5 of the boundary (the
    oracle's margin decides)."""
    w = synth.workload("c2", m=8192)
    h = _run(bfm, w, w["Y"])
    s = _run(bfm, w, w["Y"], algo=STREAM)
    ref = oracle.monitor(w["dates"], w["Y"], k=3, f=23.0, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"])
    assert (h["status"] == s["status"]).all()
    untied = ref["margin"] >= 1e-5
    assert (h["break_idx"][untied] == s["break_idx"][untied]).all()


def test_unsupported_layouts_are_refused(bfm):
    """Rows that are not a multiple of 16 bytes, and a residual ring that does
    not fit one SM's shared memory, give BFM_EUNSUPPORTED."""
    w = synth.workload("c1", m=1000)
    d = bfm.Design(w["dates"], 3, 23.0)
    Yd = torch.from_numpy(np.ascontiguousarray(w["Y"][:, :1001 - 2])).cuda()   # 999 floats per row
    with pytest.raises(bfm.BfmError) as ei:
        bfm.monitor(d, Yd, n_hist=w["n_hist"], h_frac=0.25, lam=w["lam"], algo=HYBRID)
    assert ei.value.code == 6
    w2 = synth.workload("c1", m=1024)
    N = 1200
    dates = np.arange(1, N + 1, dtype=np.float64)
    d2 = bfm.Design(dates, 3, 23.0)
    Y2 = torch.zeros((N, 1024), dtype=torch.float32, device="cuda")
    with pytest.raises(bfm.BfmError) as ei:
        bfm.monitor(d2, Y2, n_hist=1000, h_frac=1.0, lam=w2["lam"], algo=HYBRID)
    assert ei.value.code == 6
