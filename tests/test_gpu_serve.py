"""Serving loop: continuous admission under an HBM budget, concurrent
requests, device-resident results, cancellation, refusals."""
import time

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


def _tiles(count=12, scale=0.01):
    out = []
    for t in synth.tiles_c4(seed=11, count=count, scale=scale):
        d, Y, _ = synth.scene(seed=t["seed"], m=t["m"], N=t["N"], n_hist=t["n_hist"], f=23.0, k_gen=t["k"],
                              intercept=0.5, slope=0.0, coef_umax=0.3, noise_sd=0.04, miss="markov", p_a=t["p_a"],
                              p_b=t["p_b"], break_frac=0.15, step=(-0.5, -0.1),
                              dtype="i16" if t["tile"] % 3 else "f32")
        out.append(dict(t, dates=d, Y=Y, lam=synth.lambda_for_horizon(t["N"] / t["n_hist"])))
    return out


def _same(a, b):
    for key in a:
        np.testing.assert_array_equal(a[key].cpu().numpy().view(np.uint8), b[key].cpu().numpy().view(np.uint8))


def test_each_result_is_the_same_alone_and_in_the_mix(bfm):
    """Every request alone (one at a time) vs all submitted at once (host
    inputs, 4 slots, overlapping on the device): identical outputs."""
    tiles = _tiles()
    designs = [bfm.Design(t["dates"], t["k"], 23.0) for t in tiles]
    hosts = [torch.from_numpy(t["Y"]).pin_memory() for t in tiles]
    srv = bfm.Server(hbm_budget=1 << 30, slots=4)
    alone = []
    for t, d, Yh in zip(tiles, designs, hosts):
        k = srv.submit(d, Yh, n_hist=t["n_hist"], h_frac=0.25, lam=t["lam"])
        srv.wait_all(60)
        assert srv.poll(k)[0] == "done"
        alone.append(srv.result(k, d.K, t["m"]))
        srv.release(k)
    tickets = [srv.submit(d, Yh, n_hist=t["n_hist"], h_frac=0.25, lam=t["lam"])
               for t, d, Yh in zip(tiles, designs, hosts)]
    srv.wait_all(60)
    for t, d, k, a in zip(tiles, designs, tickets, alone):
        st, lat, rc = srv.poll(k)
        assert st == "done" and rc == 0 and lat > 0
        _same(srv.result(k, d.K, t["m"]), a)
        srv.release(k)
    s = srv.stats()
    assert s["completed"] == 2 * len(tiles) and s["p99_ms"] >= s["p50_ms"] > 0
    srv.close()
    # and the same as a direct bfm_monitor call
    for t, d, a in zip(tiles[:3], designs[:3], alone[:3]):
        o = bfm.monitor(d, torch.from_numpy(t["Y"]).cuda(), n_hist=t["n_hist"], h_frac=0.25, lam=t["lam"])
        torch.cuda.synchronize()
        _same(o, a)


def test_admission_waits_for_memory(bfm):
    """A budget that fits about two requests: all complete, results device-resident
    until released, later requests admitted as memory frees up."""
    tiles = _tiles(count=6, scale=0.004)
    designs = [bfm.Design(t["dates"], t["k"], 23.0) for t in tiles]
    ys = [torch.from_numpy(t["Y"]).cuda() for t in tiles]
    need = max(t["m"] * (13 + 4 * (2 + 2 * t["k"])) for t in tiles) + 8192
    srv = bfm.Server(hbm_budget=int(2.2 * need), slots=4)
    tickets = [srv.submit(d, Y, n_hist=t["n_hist"], h_frac=0.25, lam=t["lam"]) for t, d, Y in zip(tiles, designs, ys)]
    done = set()
    deadline = time.time() + 60
    while len(done) < len(tickets) and time.time() < deadline:
        for k in tickets:
            if k not in done and srv.poll(k)[0] == "done":
                srv.release(k)      # frees memory for the next admissions
                done.add(k)
        time.sleep(0.01)
    assert len(done) == len(tickets)
    srv.close()


def test_refusals_and_cancellation(bfm):
    tiles = _tiles(count=4, scale=0.01)
    d = bfm.Design(tiles[0]["dates"], tiles[0]["k"], 23.0)
    Y = torch.from_numpy(tiles[0]["Y"]).cuda()
    small = bfm.Server(hbm_budget=4096, slots=1)  # smaller than any request's outputs
    assert tiles[0]["m"] >= 100
    with pytest.raises(bfm.BfmError) as ei:
        small.submit(d, Y, n_hist=tiles[0]["n_hist"], h_frac=0.25, lam=1.7)
    assert ei.value.code == 5  # BFM_EBUSY: larger than the whole budget
    small.close()
    with pytest.raises(bfm.BfmError) as ei:
        bfm.Server(hbm_budget=1 << 50, slots=1)  # more than the device has
    assert ei.value.code == 2  # BFM_ENOMEM
    srv = bfm.Server(hbm_budget=1 << 28, slots=1)
    ks = [srv.submit(d, Y, n_hist=tiles[0]["n_hist"], h_frac=0.25, lam=1.7) for _ in range(6)]
    cancelled = 0
    for k in ks[2:]:
        try:
            srv.cancel(k)
            cancelled += 1
        except bfm.BfmError:
            pass
    srv.wait_all(60)
    states = [srv.poll(k)[0] for k in ks]
    assert states.count("cancelled") == cancelled and states.count("done") == len(ks) - cancelled
    ref = srv.result(ks[0], d.K, tiles[0]["m"])
    for k, st in zip(ks, states):
        if st == "done":
            _same(srv.result(k, d.K, tiles[0]["m"]), ref)
    srv.close()


def test_explicit_forms_and_bad_algo(bfm):
    """A request with an explicit form: the complete-series form on a cloud-free tile equals a direct
    bfm_monitor call with that form; an algo outside the bfm_algo values is refused at submit."""
    d_, Y, _ = synth.scene(seed=31, m=2048, N=228, n_hist=100, f=23.0, k_gen=2, intercept=0.5, slope=0.001,
                           coef_fixed=[0.2, 0.0, 0.0, 0.05], noise_sd=0.03, miss="none", break_frac=0.2,
                           step=(-0.3, -0.3), dtype="f32")
    d = bfm.Design(d_, 3, 23.0)
    Yd = torch.from_numpy(Y).cuda()
    lam = synth.workload_lambda("c1")
    srv = bfm.Server(hbm_budget=1 << 28, slots=2)
    for algo in (bfm.BFM_ALGO_COMPLETE, bfm.BFM_ALGO_STREAM, bfm.BFM_ALGO_SIMT):
        k = srv.submit(d, Yd, n_hist=100, h_frac=0.25, lam=lam, algo=algo)
        srv.wait_all(60)
        st, _, rc = srv.poll(k)
        assert st == "done" and rc == 0
        direct = bfm.monitor(d, Yd, n_hist=100, h_frac=0.25, lam=lam, algo=algo)
        torch.cuda.synchronize()
        _same(srv.result(k, d.K, 2048), direct)
        srv.release(k)
    with pytest.raises(bfm.BfmError) as ei:
        srv.submit(d, Yd, n_hist=100, h_frac=0.25, lam=lam, algo=7)
    assert ei.value.code == 1
    srv.close()
