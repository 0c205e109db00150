"""The failure path of the bounded waits, made to run on purpose.

Every wait of the library's kernels is bounded, so that a copy that never
lands ends the kernel with an error status instead of hanging the GPU.  Here
the consumer-side stage wait of the staged forms is shortened (bfm_stage_wait_limit)
until it gives up at the first stage that has not landed yet: the kernel must
end, set bit 0 of the device error word, mark the unfinished pixels
BFM_PX_TIMEOUT with the unfitted outputs, and leave the context usable, so
that the next run with the default bound matches the oracle.
"""
import numpy as np
import pytest

import synth
from _parity import compare, to_numpy

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STREAM, HYBRID = 4, 5
TIMEOUT = 255


@pytest.fixture(scope="module")
def bfm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_01751_gb300 as bfm
    bfm.load()
    return bfm


@pytest.mark.parametrize("algo", [STREAM, HYBRID], ids=["stream", "hybrid"])
@pytest.mark.parametrize("name", ["c1", "c3"])
def test_stage_wait_runs_out_then_recovers(bfm, name, algo):
    w = synth.workload(name, m=4096)
    d = bfm.Design(w["dates"], w["k"], w["f"])
    Yd = torch.from_numpy(np.ascontiguousarray(w["Y"])).cuda()
    kw = dict(n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"], algo=algo)
    assert bfm.bfm_device_errors() == 0
    bfm.bfm_stage_wait_limit(1)          # one look at each stage barrier, no waiting
    try:
        short = to_numpy(bfm.monitor(d, Yd, **kw))
        torch.cuda.synchronize()
        bits = bfm.bfm_device_errors()
    finally:
        bfm.bfm_stage_wait_limit(0)      # back to the default bound
    assert bits & 1
    timed = short["status"] == TIMEOUT
    assert timed.sum() > 0
    assert (short["break_idx"][timed] == -1).all()
    assert np.isnan(short["sigma"][timed]).all() and np.isnan(short["beta"][:, timed]).all()
    normal = to_numpy(bfm.monitor(d, Yd, **kw))
    torch.cuda.synchronize()
    assert bfm.bfm_device_errors() == 0
    # pixels the short-bound run finished are exactly the normal run's
    for key in normal:
        a, b = short[key][..., ~timed], normal[key][..., ~timed]
        np.testing.assert_array_equal(a.view(np.uint8), b.view(np.uint8))
    ref = oracle.monitor(w["dates"], w["Y"], k=w["k"], f=w["f"], n_hist=w["n_hist"], h_frac=w["h_frac"],
                         lam=w["lam"])
    rep = compare(normal, ref, w["dates"], w["k"], w["f"], tol=1e-5)
    assert rep["ok"], rep
