"""The seeded scene generator: determinism, prefix stability, statistics."""
import numpy as np

import synth


def test_dates_strictly_increasing_with_jitter():
    d = synth.dates(2, 414)
    assert np.all(np.diff(d) > 0)
    i = np.arange(1, 415)
    assert np.all(np.abs(d * 16 - 16 * i) <= 3)


def test_scene_deterministic_and_prefix_stable():
    a = synth.workload("c1", m=1000)
    b = synth.workload("c1", m=3000)
    np.testing.assert_array_equal(a["Y"], b["Y"][:, :1000])
    np.testing.assert_array_equal(a["true_break"], b["true_break"][:1000])


def test_missing_fractions():
    c1 = synth.workload("c1", m=4096)
    assert abs(np.isnan(c1["Y"]).mean() - 0.3) < 0.01
    c2 = synth.workload("c2", m=20000)
    assert abs(np.isnan(c2["Y"]).mean() - 0.6) < 0.02
    assert abs((c2["true_break"] >= 0).mean() - 0.1) < 0.01
    c3 = synth.workload("c3", m=4096)
    assert c3["Y"].dtype == np.int16
    np.testing.assert_array_equal(c3["Y"] == -32768, np.isnan(c1["Y"]))
    ok = ~np.isnan(c1["Y"])
    assert np.abs(c3["Y"][ok] - np.round(c1["Y"][ok].astype(np.float64) * 1e4)).max() <= 1
