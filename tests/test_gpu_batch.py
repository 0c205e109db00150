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


def _mask_bits(rng, N, m, p_keep=0.85):
    words = (m + 31) // 32
    keep = rng.random((N, words * 32)) < p_keep
    bits = np.zeros((N, words), np.uint32)
    for b in range(32):
        bits |= keep[:, b::32].astype(np.uint32) << np.uint32(b)
    return torch.from_numpy(bits.view(np.int32)).cuda()


def test_batch_tensor_core_variants(bfm):
    """Tiles of every harmonic order in both storage types, widths rounded to
    multiples of 8, in a batch limited to the tensor-core form: the tile nodes
    of the graph reproduce single calls bit for bit, on two replays."""
    tiles = _tiles(scale=0.02, count=16, px_multiple=8)
    b = bfm.Batch(forms=bfm.BFM_ALGO_MMA)
    outs, singles, forms = [], [], set()
    for i, t in enumerate(tiles):
        d = bfm.Design(t["dates"], t["k"], 23.0)
        Yd = torch.from_numpy(t["Y"]).cuda()
        dt = bfm.BFM_F32 if t["Y"].dtype == np.float32 else bfm.BFM_I16
        outs.append(b.add(d, Yd, n_hist=t["n_hist"], h_frac=0.25, lam=t["lam"]))
        form = b.form(i)
        assert form in (bfm.BFM_ALGO_MMA, bfm.BFM_ALGO_SIMT)
        if form == bfm.BFM_ALGO_MMA:
            forms.add((t["k"], dt))
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


def test_batch_hybrid_variants(bfm):
    """Tiles of every harmonic order in both storage types, some with mask
    bits, in a batch of the default forms: the hybrid form takes the tiles
    whose tables and ring fit one SM; its persistent kernels (one per variant
    and layout group, tables reloaded where a CTA's next block belongs to
    another tile) reproduce single calls bit for bit, on two replays."""
    tiles = _tiles(scale=0.02, count=16, px_multiple=8)
    rng = np.random.default_rng(11)
    b = bfm.Batch()
    outs, singles, forms = [], [], {}
    for i, t in enumerate(tiles):
        d = bfm.Design(t["dates"], t["k"], 23.0)
        Yd = torch.from_numpy(t["Y"]).cuda()
        dt = bfm.BFM_F32 if t["Y"].dtype == np.float32 else bfm.BFM_I16
        mb = _mask_bits(rng, t["N"], t["m"]) if i % 4 == 1 else None
        outs.append(b.add(d, Yd, n_hist=t["n_hist"], h_frac=0.25, lam=t["lam"], mask_bits=mb))
        form = b.form(i)
        assert form == bfm.bfm_batch_form(d, dt, t["n_hist"], 0.25, Yd, t["m"])
        v = (t["k"], dt, mb is not None)
        forms[v] = forms.get(v, 0) + (form == bfm.BFM_ALGO_HYBRID)
        singles.append(bfm.monitor(d, Yd, n_hist=t["n_hist"], h_frac=0.25, lam=t["lam"], mask_bits=mb, algo=form))
    assert sum(1 for v in forms.values() if v) >= 4, forms
    b.run()
    b.run()
    torch.cuda.synchronize()
    assert bfm.bfm_device_errors() == 0
    for i, (o, sgl) in enumerate(zip(outs, singles)):
        a, c = to_numpy(o), to_numpy(sgl)
        for key in a:
            np.testing.assert_array_equal(a[key].view(np.uint8), c[key].view(np.uint8), err_msg=f"tile {i} {key}")
    b.close()


def test_batch_hybrid_groups_of_one_variant(bfm):
    """Two float k = 3 tiles whose shared-memory layouts fit one SM alone but
    not together (226.5 KB and 217.3 KB; 236.7 KB as one layout): the batch
    runs them as two hybrid groups of the same kernel variant with different
    shared-memory sizes, in one graph, and both reproduce single calls bit for
    bit."""
    b = bfm.Batch()
    outs, singles = [], []
    for i, (N, n_hist) in enumerate(((414, 228), (600, 200))):
        d_, Y, _ = synth.scene(seed=40 + i, m=2048, N=N, n_hist=n_hist, f=23.0, k_gen=3, intercept=0.5, slope=0.0,
                               coef_umax=0.3, noise_sd=0.04, miss="markov", p_a=0.25, p_b=0.375, break_frac=0.15,
                               step=(-0.5, -0.1), dtype="f32")
        d = bfm.Design(d_, 3, 23.0)
        Yd = torch.from_numpy(Y).cuda()
        lam = synth.lambda_for_horizon(N / n_hist)
        outs.append(b.add(d, Yd, n_hist=n_hist, h_frac=0.25, lam=lam))
        assert b.form(i) == bfm.BFM_ALGO_HYBRID
        singles.append(bfm.monitor(d, Yd, n_hist=n_hist, h_frac=0.25, lam=lam, algo=bfm.BFM_ALGO_HYBRID))
    b.run()
    b.run()
    torch.cuda.synchronize()
    assert bfm.bfm_device_errors() == 0
    for i, (o, sgl) in enumerate(zip(outs, singles)):
        a, c = to_numpy(o), to_numpy(sgl)
        for key in a:
            np.testing.assert_array_equal(a[key].view(np.uint8), c[key].view(np.uint8), err_msg=f"tile {i} {key}")
    b.close()


def test_batch_forms_api(bfm):
    """bfm_batch_set_forms takes AUTO, HYBRID, MMA or SIMT before the first
    tile only; bfm_batch_tile_form answers -1 for an unknown id."""
    b = bfm.Batch()
    with pytest.raises(bfm.BfmError):
        bfm.bfm_batch_set_forms(b.handle, bfm.BFM_ALGO_STREAM)
    bfm.bfm_batch_set_forms(b.handle, bfm.BFM_ALGO_SIMT)
    t = _tiles(count=1)[0]
    d = bfm.Design(t["dates"], t["k"], 23.0)
    b.add(d, torch.from_numpy(t["Y"]).cuda(), n_hist=t["n_hist"], h_frac=0.25, lam=t["lam"])
    assert b.form(0) == bfm.BFM_ALGO_SIMT
    assert bfm.bfm_batch_tile_form(b.handle, 1) == -1
    with pytest.raises(bfm.BfmError):
        bfm.bfm_batch_set_forms(b.handle, bfm.BFM_ALGO_AUTO)
    b.close()


def test_batch_descriptors_at_reused_addresses(bfm):
    """Batches created and destroyed in turn, over different tile sets: each
    batch's tensor maps land in device memory that earlier batches' maps
    occupied, and the TMA unit must not use a stale copy of a map at a reused
    address.  Every batch reproduces single calls bit for bit."""
    sets = []
    for tiles in (_tiles(scale=0.02, count=8, px_multiple=8), _tiles(scale=0.01, count=8)):
        row = []
        for t in tiles:
            d = bfm.Design(t["dates"], t["k"], 23.0)
            row.append((d, torch.from_numpy(t["Y"]).cuda(), t))
        sets.append(row)
    refs = {}  # (set, tile, form) -> single-call outputs
    for it in range(8):
        si, forms = it % 2, (bfm.BFM_ALGO_AUTO, bfm.BFM_ALGO_MMA)[(it // 2) % 2]
        b = bfm.Batch(forms=forms)
        outs = [b.add(d, Yd, n_hist=t["n_hist"], h_frac=0.25, lam=t["lam"]) for d, Yd, t in sets[si]]
        b.run()
        torch.cuda.synchronize()
        assert bfm.bfm_device_errors() == 0
        for i, (o, (d, Yd, t)) in enumerate(zip(outs, sets[si])):
            key = (si, i, b.form(i))
            if key not in refs:
                refs[key] = to_numpy(bfm.monitor(d, Yd, n_hist=t["n_hist"], h_frac=0.25, lam=t["lam"], algo=key[2]))
            a = to_numpy(o)
            for k in a:
                np.testing.assert_array_equal(a[k].view(np.uint8), refs[key][k].view(np.uint8), err_msg=f"{it} {i} {k}")
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
