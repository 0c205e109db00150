"""bfm_batch_run_static: the batch entry point that allocates nothing.

Callers that cannot allocate device memory while they run work (a serving
process whose memory is pre-reserved by its own pool, a latency-critical
loop where cudaMalloc/cudaFree would synchronise the device) use this entry
point; its tile table, tensor maps and work counter live in a fixed array
inside the library.  Its outputs must equal those of the ordinary entry
point (bfm_monitor, CUDA-core form) on every tile, on calls in a row that
share and overwrite that array (four calls, alternating two tile sets).
This file is collected last.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bfm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_01751_gb300 as bfm
    bfm.load()
    return bfm


def _tiles(seed, count):
    out = []
    for t in synth.tiles_c4(seed=seed, count=count, scale=0.005):
        d, Y, _ = synth.scene(seed=t["seed"], m=t["m"], N=t["N"], n_hist=t["n_hist"], f=23.0, k_gen=t["k"],
                              intercept=0.5, slope=0.0, coef_umax=0.3, noise_sd=0.04, miss="markov", p_a=t["p_a"],
                              p_b=t["p_b"], break_frac=0.15, step=(-0.5, -0.1),
                              dtype="i16" if t["tile"] % 2 else "f32")
        out.append(dict(t, dates=d, Y=Y, lam=synth.lambda_for_horizon(t["N"] / t["n_hist"])))
    return out


def _run_and_compare(bfm, tiles):
    specs, outs, refs, keep = [], [], [], []
    for t in tiles:
        d = bfm.Design(t["dates"], t["k"], 23.0)
        Yd = torch.from_numpy(t["Y"]).cuda()
        o = bfm.empty_outputs(d.K, Yd.shape[1])
        specs.append(bfm.tile_spec(d, Yd, n_hist=t["n_hist"], h_frac=0.25, lam=t["lam"], out=o))
        refs.append(bfm.monitor(d, Yd, n_hist=t["n_hist"], h_frac=0.25, lam=t["lam"], algo=bfm.BFM_ALGO_SIMT))
        outs.append(o)
        keep.append((d, Yd))
    bfm.bfm_batch_run_static(specs)
    torch.cuda.synchronize()
    assert bfm.bfm_device_errors() == 0
    for o, r in zip(outs, refs):
        for key in o:
            a, b = o[key].cpu().numpy(), r[key].cpu().numpy()
            # identical arithmetic: equal bit for bit (NaN where the other is NaN)
            np.testing.assert_array_equal(a.view(np.uint8), b.view(np.uint8))
    return outs


def test_static_entry_matches_ordinary_entry_two_calls(bfm):
    first = _tiles(seed=7, count=12)
    second = _tiles(seed=8, count=5)   # fewer tiles: stale entries of the first call must not matter
    # each call rewrites the tensor maps at the same addresses: alternating
    # calls fail if the TMA unit used a cached copy of an earlier call's map
    for tiles in (first, second, first, second):
        _run_and_compare(bfm, tiles)


def test_static_entry_rejects_too_many_tiles(bfm):
    t = _tiles(seed=9, count=1)[0]
    d = bfm.Design(t["dates"], t["k"], 23.0)
    Yd = torch.from_numpy(t["Y"]).cuda()
    o = bfm.empty_outputs(d.K, Yd.shape[1])
    spec = bfm.tile_spec(d, Yd, n_hist=t["n_hist"], h_frac=0.25, lam=t["lam"], out=o)
    with pytest.raises(bfm.BfmError) as ei:
        bfm.bfm_batch_run_static([spec] * (bfm.BFM_STATIC_MAX_TILES + 1))
    assert ei.value.code == 1 and "maximum" in str(ei.value)
