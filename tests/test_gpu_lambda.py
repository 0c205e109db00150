"""Critical value lambda(alpha, h, N/n) of Eq. 4 simulated on the GPU
(bfm_lambda) against the oracle's simulation of the same process.

Both sides draw every path from its own SplitMix64 stream with Box-Muller
normals and accumulate W in FP64 in the same order, so the per-path
statistics agree up to the last-ulp differences of log and cos between the
CUDA and host math libraries; lambda is then the same order statistic.
"""
import json
import os

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def bfm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_01751_gb300 as bfm
    bfm.load()
    return bfm


@pytest.mark.parametrize("alpha,h,T,G", [(0.05, 0.25, 1.816, 400), (0.05, 0.5, 2.0, 300), (0.01, 0.25, 2.28, 250),
                                         (0.1, 1.0, 1.5, 200)])
def test_paths_match_oracle(bfm, alpha, h, T, G):
    reps = 4000
    lam_g, st_g = bfm.bfm_lambda(alpha, h, T, G=G, reps=reps, seed=7, return_stats=True)
    lam_o, st_o = oracle.critical_value(alpha, h, T, G=G, reps=reps, seed=7, return_stats=True)
    rel = np.abs(st_g - st_o) / np.maximum(np.abs(st_o), 1e-300)
    print("max relative difference of the path statistics", rel.max())
    assert rel.max() < 1e-9
    assert abs(lam_g - lam_o) <= 1e-9 * lam_o


def test_paper_value(bfm):
    """Section 4.3: 2.39 for alpha = 0.05, h/n = 0.5, N/n = 2 (weak pin, as for
    the oracle: the paper does not state its grid or replicate counts)."""
    with open(os.path.join(GOLDEN, "paper_values.json")) as fh:
        g = json.load(fh)["critical_value_chile"]
    lam = bfm.bfm_lambda(g["alpha"], g["h_over_n"], g["N_over_n"], G=800, reps=100000, seed=3)
    print("lambda", lam)
    assert abs(lam - g["lambda"]) < g["tolerance"]


def test_invalid_arguments(bfm):
    for args in ((0.0, 0.5, 2.0), (1.0, 0.5, 2.0), (0.05, 0.0, 2.0), (0.05, 1.5, 2.0), (0.05, 0.5, 1.0)):
        with pytest.raises(bfm.BfmError) as ei:
            bfm.bfm_lambda(*args, G=100, reps=10)
        assert ei.value.code == 1
    with pytest.raises(bfm.BfmError):
        bfm.bfm_lambda(0.05, 0.001, 2.0, G=100, reps=10)  # h * G rounds to 0
