"""Batched persistent launch (one CUDA-graph replay over tiles of uneven
pixel counts, series lengths, harmonics and storage types)."""
import numpy as np
import pytest

import oracle
import synth
from _parity import compare, to_numpy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bfm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_01751_gb300 as bfm
    bfm.load()
    return bfm


def _tiles(scale=0.01, count=10, px_multiple=1):
    out = []
    for t in synth.tiles_c4(seed=4, count=count, scale=scale, px_multiple=px_multiple):
        d, Y, _ = synth.scene(seed=t["seed"], m=t["m"], N=t["N"], n_hist=t["n_hist"], f=23.0, k_gen=t["k"],
                              intercept=0.5, slope=0.0, coef_umax=0.3, noise_sd=0.04, miss="markov", p_a=t["p_a"],
                              p_b=t["p_b"], break_frac=0.15, step=(-0.5, -0.1),
                              dtype="i16" if t["tile"] % 3 else "f32")
        lam = synth.lambda_for_horizon(t["N"] / t["n_hist"])
        out.append(dict(t, dates=d, Y=Y, lam=lam))
    return out


def test_batch_equals_single_calls_and_oracle(bfm):
    tiles = _tiles()
    b = bfm.Batch()
    outs, singles = [], []
    for t in tiles:
        d = bfm.Design(t["dates"], t["k"], 23.0)
        Yd = torch.from_numpy(t["Y"]).cuda()
        outs.append(b.add(d, Yd, n_hist=t["n_hist"], h_frac=0.25, lam=t["lam"]))
        dt = bfm.BFM_F32 if t["Y"].dtype == np.float32 else bfm.BFM_I16
        form = bfm.bfm_batch_form(d, dt, t["n_hist"], 0.25, Yd, t["m"])
        singles.append(bfm.monitor(d, Yd, n_hist=t["n_hist"], h_frac=0.25, lam=t["lam"], algo=form))
    b.run()
    torch.cuda.synchronize()
    assert bfm.bfm_device_errors() == 0
    for t, o, s in zip(tiles, outs, singles):
        a, c = to_numpy(o), to_numpy(s)
        for key in a:
            np.testing.assert_array_equal(a[key].view(np.uint8), c[key].view(np.uint8))
    # oracle on every tile (first 512 pixels)
    for t, o in zip(tiles, outs):
        g = {k: (v[:, :512] if v.dim() == 2 else v[:512]).cpu().numpy() for k, v in o.items()}
        Ys = t["Y"][:, :512]
        ref = oracle.monitor(t["dates"], Ys, k=t["k"], f=23.0, n_hist=t["n_hist"], h_frac=0.25, lam=t["lam"])
        rep = compare(g, ref, t["dates"], t["k"], 23.0, tol=1e-5 if t["Y"].dtype == np.float32 else 1e-4)
        assert rep["ok"], (t["tile"], rep)
    b.close()


def test_batch_tensor_core_variants(bfm):
    """Tiles of every harmonic order in both storage types, widths rounded to
    multiples of 8 so that the batch gives them the tensor-core form: the
    persistent tensor-core kernels (one per variant) reproduce single calls
    bit for bit."""
    tiles = _tiles(scale=0.02, count=16, px_multiple=8)
    b = bfm.Batch()
    outs, singles, forms = [], [], set()
    for t in tiles:
        d = bfm.Design(t["dates"], t["k"], 23.0)
        Yd = torch.from_numpy(t["Y"]).cuda()
        dt = bfm.BFM_F32 if t["Y"].dtype == np.float32 else bfm.BFM_I16
        form = bfm.bfm_batch_form(d, dt, t["n_hist"], 0.25, Yd, t["m"])
        if form == bfm.BFM_ALGO_MMA:
            forms.add((t["k"], dt))
        outs.append(b.add(d, Yd, n_hist=t["n_hist"], h_frac=0.25, lam=t["lam"]))
        singles.append(bfm.monitor(d, Yd, n_hist=t["n_hist"], h_frac=0.25, lam=t["lam"], algo=form))
    assert len(forms) >= 4, forms
    b.run()
    b.run()
    torch.cuda.synchronize()
    assert bfm.bfm_device_errors() == 0
    for o, sgl in zip(outs, singles):
        a, c = to_numpy(o), to_numpy(sgl)
        for key in a:
            np.testing.assert_array_equal(a[key].view(np.uint8), c[key].view(np.uint8))
    b.close()


def test_batch_graph_replay_and_autotune_keep_results(bfm):
    tiles = _tiles(count=6)
    b = bfm.Batch()
    outs = []
    for t in tiles:
        d = bfm.Design(t["dates"], t["k"], 23.0)
        outs.append(b.add(d, torch.from_numpy(t["Y"]).cuda(), n_hist=t["n_hist"], h_frac=0.25, lam=t["lam"]))
    b.run()
    torch.cuda.synchronize()
    first = [to_numpy(o) for o in outs]
    for o in outs:
        for v in o.values():
            v.zero_()
    cps, grab, ms = b.autotune()
    assert cps >= 1 and grab in (1, 2, 4, 8) and ms > 0
    b.run()
    b.run()
    torch.cuda.synchronize()
    for a, o in zip(first, outs):
        c = to_numpy(o)
        for key in a:
            np.testing.assert_array_equal(a[key].view(np.uint8), c[key].view(np.uint8))
    b.close()


def test_batch_empty_and_zero_pixel_tiles(bfm):
    b = bfm.Batch()
    b.run()  # nothing to do
    t = _tiles(count=2)
    d = bfm.Design(t[0]["dates"], t[0]["k"], 23.0)
    Y0 = torch.empty((t[0]["N"], 0), dtype=torch.float32, device="cuda")
    b.add(d, Y0, n_hist=t[0]["n_hist"], h_frac=0.25, lam=1.7)
    o = b.add(d, torch.from_numpy(t[0]["Y"]).cuda(), n_hist=t[0]["n_hist"], h_frac=0.25, lam=1.7)
    b.run()
    torch.cuda.synchronize()
    assert (o["status"].cpu().numpy() <= 4).all()
    b.close()
