"""Pins of the FP64 oracle to things other than itself.

Each test ties a part of the oracle to a closed form, a library routine, an
invariant of the method, or a value printed in the paper, chosen so that a
plausible slip (wrong window length, sqrt(h) instead of sqrt(n), wrong
degrees of freedom, sign, off-by-one in positions, transposed design) fails.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dates_regular(N):
    return np.arange(1, N + 1, dtype=np.float64)


def _design_np(d, k, f):
    # independent construction with numpy for the regressor layout of Eq. 2
    cols = [np.ones_like(d), d]
    for j in range(1, k + 1):
        cols += [np.sin(2 * np.pi * j * d / f), np.cos(2 * np.pi * j * d / f)]
    return np.stack(cols, axis=1)


# ---------------------------------------------------------------- design ----

def test_design_special_values():
    """Eq. 2 at dates with known sines/cosines: t = f/4 gives sin F(1) = 1,
    cos F(1) = 0, sin F(2) = 0, cos F(2) = -1, sin F(3) = -1, cos F(3) = 0."""
    f = 23.0
    X = oracle.design(np.array([f / 4, f / 2]), 3, f)
    assert X.shape == (2, 8)
    np.testing.assert_allclose(X[0], [1, f / 4, 1, 0, 0, -1, -1, 0], atol=1e-15)
    np.testing.assert_allclose(X[1], [1, f / 2, 0, -1, 0, 1, 0, -1], atol=1e-14)


def test_design_pythagoras_and_layout():
    d = synth.dates(7, 50)
    X = oracle.design(d, 3, 23.0)
    for j in range(3):
        np.testing.assert_allclose(X[:, 2 + 2 * j] ** 2 + X[:, 3 + 2 * j] ** 2, 1.0, atol=1e-15)
    np.testing.assert_array_equal(X[:, 0], 1.0)
    np.testing.assert_array_equal(X[:, 1], d)


# ------------------------------------------------------------ least squares --

@pytest.mark.parametrize("n,K,seed", [(9, 4, 0), (12, 6, 1), (16, 8, 2), (40, 8, 3)])
def test_qr_matches_lapack_and_normal_equations(n, K, seed):
    """Householder QR vs LAPACK (numpy.linalg.lstsq, SVD based) vs the
    normal equations of Eq. 6, plus the optimality condition A'(y - A b) = 0."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, K))
    y = rng.standard_normal(n)
    b_qr, rd = oracle.lstsq_qr(A, y)
    b_np = np.linalg.lstsq(A, y, rcond=None)[0]
    b_ne = oracle.lstsq_normal(A, y)
    np.testing.assert_allclose(b_qr, b_np, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(b_ne, b_np, rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(A.T @ (y - A @ b_qr), 0.0, atol=1e-11)
    # |R_kk| from the QR agrees with the Cholesky factor of A'A
    Lc = np.linalg.cholesky(A.T @ A)
    np.testing.assert_allclose(np.abs(rd), np.diag(Lc), rtol=1e-9)


def test_qr_brute_force_tiny():
    """On a 5x2 problem the least-squares value is the minimum over a fine
    grid of candidate coefficients (brute force)."""
    A = np.array([[1, 0.0], [1, 1], [1, 2], [1, 3], [1, 4]])
    y = np.array([0.1, 0.9, 2.2, 2.8, 4.1])
    b, _ = oracle.lstsq_qr(A, y)
    best = min(((y - A @ np.array([a0, a1])) ** 2).sum()
               for a0 in np.linspace(-0.5, 0.5, 201) for a1 in np.linspace(0.5, 1.5, 201))
    assert ((y - A @ b) ** 2).sum() <= best + 1e-12
    # closed form of the simple linear regression
    xb, yb = 2.0, y.mean()
    slope = ((A[:, 1] - xb) * (y - yb)).sum() / ((A[:, 1] - xb) ** 2).sum()
    np.testing.assert_allclose(b, [yb - slope * xb, slope], rtol=1e-13)


# -------------------------------------------------------------- boundary ----

def test_boundary_closed_forms():
    """Eq. 4: b = lambda for t/n <= e, lambda*sqrt(log 8) = lambda*sqrt(3 ln 2)
    at t/n = 8; log+ is continuous at e."""
    lam = 1.7
    assert oracle.boundary(lam, 100, 100) == lam
    assert oracle.boundary(lam, 271, 100) == lam  # 2.71 < e
    np.testing.assert_allclose(oracle.boundary(lam, 800, 100), lam * math.sqrt(3 * math.log(2)), rtol=1e-15)
    np.testing.assert_allclose(oracle.logplus(math.e * (1 + 1e-12)), 1.0, atol=1e-11)
    assert oracle.logplus(math.e) == 1.0


# ------------------------------------------------------ full monitor path ---

def _orth_noise(Xh, rng, eps):
    """noise exactly orthogonal to the history design (LAPACK projection)."""
    e = rng.standard_normal(Xh.shape[0]) * eps
    coef = np.linalg.lstsq(Xh, e, rcond=None)[0]
    return e - Xh @ coef


def _closed_form_mosum(r, n, K, h, lam):
    """MOSUM of Eq. 3 from a KNOWN residual vector by prefix sums."""
    sig = math.sqrt((r[:n] ** 2).sum() / (n - K))
    S = np.concatenate([[0.0], np.cumsum(r)])
    N = r.size
    j = np.arange(n + 1, N + 1)
    mo = (S[j] - S[j - h]) / (sig * math.sqrt(n))
    b = np.array([lam * math.sqrt(1.0 if jj / n <= math.e else math.log(jj / n)) for jj in j])
    cross = np.nonzero(np.abs(mo) > b)[0]
    first = int(j[cross[0]] - 1) if cross.size else -1  # 0-based position
    return sig, mo, first


@pytest.mark.parametrize("k,missing", [(3, False), (3, True), (1, True), (2, False)])
def test_exact_fit_orthogonal_noise_and_step(k, missing):
    """History = x'beta + e with e orthogonal to the history design, so the
    OLS fit is exact (beta-hat = beta), the history residuals are e and
    sigma-hat = ||e||/sqrt(n-K); monitoring = x'beta + d after the step.
    Every MOSUM value, the break and the mean then have closed forms."""
    rng = np.random.default_rng(10 + k + 2 * missing)
    N, n_hist, f, lam, hf = 160, 70, 23.0, 1.8, 0.25
    d = synth.dates(3, N)
    K = 2 + 2 * k
    valid = np.ones(N, bool)
    if missing:
        valid = rng.random(N) > 0.3
        valid[0] = valid[n_hist] = True
    idx = np.nonzero(valid)[0]
    n = int((idx < n_hist).sum())
    X = _design_np(d[idx], k, f)
    beta = rng.uniform(-0.3, 0.3, K)
    beta[0], beta[1] = 0.5, 0.002
    e = _orth_noise(X[:n], rng, 0.02)
    j0 = n + 25  # 0-based valid position of the step
    dstep = -0.4
    r_true = np.concatenate([e, np.where(np.arange(n, idx.size) >= j0, dstep, 0.0)])
    y = X @ beta + r_true
    Y = np.full((N, 1), np.nan)
    Y[idx, 0] = y
    o = oracle.monitor(d, Y, k=k, f=f, n_hist=n_hist, h_frac=hf, lam=lam, trace=True)
    h = max(1, min(int(math.floor(hf * n)), n))
    sig, mo, first = _closed_form_mosum(r_true, n, K, h, lam)
    np.testing.assert_allclose(o["beta"][:, 0], beta, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(o["sigma"][0], sig, rtol=1e-10)
    assert o["n"][0] == n and o["Nv"][0] == idx.size and o["h"][0] == h
    tr = o["mo_trace"][0, : idx.size - n]
    np.testing.assert_allclose(tr, mo, rtol=1e-8, atol=1e-9)
    assert first == j0  # the step is far above the boundary
    assert o["break_idx"][0] == idx[first]
    np.testing.assert_allclose(o["mean_mosum"][0], mo.mean(), rtol=1e-9)
    assert o["status"][0] == 0


def test_noise_free_series_recovered_exactly():
    """A noise-free harmonic series: beta to 1e-12, sigma-hat ~ 0, status
    DEGENERATE (MO = 0, no break, mean 0), also with missing values."""
    N, n_hist, f = 120, 60, 23.0
    d = synth.dates(5, N)
    X = _design_np(d, 3, f)
    beta = np.array([0.6, -0.001, 0.2, 0.1, -0.05, 0.03, 0.01, -0.02])
    Y = np.stack([X @ beta, X @ beta], axis=1)
    Y[::3, 1] = np.nan
    o = oracle.monitor(d, Y, k=3, f=f, n_hist=n_hist, h_frac=0.25, lam=1.7)
    for p in range(2):
        np.testing.assert_allclose(o["beta"][:, p], beta, rtol=1e-12, atol=1e-13)
        assert o["sigma"][p] < 1e-13
        assert o["status"][p] == 3 and o["break_idx"][p] == -1 and o["mean_mosum"][p] == 0.0


def test_window_sums_are_cumsum_differences_on_complete_series():
    """Complete series: every MOSUM value of Eq. 3 is a difference of the
    cumulative residual sum, (S_j - S_{j-h}) / (sigma-hat sqrt(n)), with
    S_j = r_1 + ... + r_j, h = floor(0.25 n) terms per window and sigma-hat
    from the n history residuals with n - (2 + 2k) degrees of freedom
    (Section 2.1).  The oracle forms each window by a direct sum instead."""
    w = synth.workload("c1", m=64)
    N, n, k, f = w["N"], w["n_hist"], 3, w["f"]
    _, Yc, _ = synth.scene(seed=11, m=64, N=N, n_hist=n, f=f, dtype="f32", k_gen=2, intercept=0.5,
                           slope=0.001, coef_fixed=[0.2, 0.0, 0.0, 0.05], noise_sd=0.03, miss="none",
                           break_frac=0.3, step=(-0.3, -0.3), date_vals=w["dates"])
    Yd = Yc.astype(np.float64)
    o = oracle.monitor(w["dates"], Yd, k=k, f=f, n_hist=n, h_frac=0.25, lam=w["lam"], trace=True)
    X = _design_np(w["dates"], k, f)
    h = int(0.25 * n)
    pos = np.arange(n + 1, N + 1)              # 1-based monitoring positions
    for p in range(0, 64, 7):
        resid = Yd[:, p] - X @ o["beta"][:, p]
        cum = np.concatenate([[0.0], np.cumsum(resid)])
        sig = math.sqrt((resid[:n] ** 2).sum() / (n - (2 + 2 * k)))
        mo = (cum[pos] - cum[pos - h]) / (sig * math.sqrt(n))
        np.testing.assert_allclose(o["mo_trace"][p, : N - n], mo, rtol=1e-9, atol=1e-10)
        np.testing.assert_allclose(o["sigma"][p], sig, rtol=1e-12)


def _residuals_for_trace(e, mo, h, K):
    """Monitoring residuals whose MOSUM process (Eq. 3) is exactly `mo`, given
    the history residuals e: with W_j = sigma-hat sqrt(n) mo_j the sum of the h
    residuals ending at position j, r_j = W_j - W_{j-1} + r_{j-h}."""
    n = e.size
    scale = math.sqrt((e ** 2).sum() / (n - K)) * math.sqrt(n)
    r = np.concatenate([e, np.zeros(mo.size)])
    w_prev = e[n - h:].sum()                    # window ending at the last history position
    for i in range(mo.size):
        j = n + i                               # 0-based index of position n + 1 + i
        w = scale * mo[i]
        r[j] = w - w_prev + r[j - h]
        w_prev = w
    return r


def _boundary_np(lam, n, npos):
    j = np.arange(n + 1, n + 1 + npos)
    return lam * np.sqrt(np.where(j / n <= math.e, 1.0, np.log(j / n)))


@pytest.mark.parametrize("case", ["min_at_break", "min_before_break", "no_break"])
def test_margin_closed_form(case):
    """The tie margin min ||MO_j| - b_j| over the monitoring positions up to and
    including the first crossing (all positions when there is none), from a
    prescribed MOSUM process: the monitoring residuals are built so that Eq. 3
    gives exactly that process (history noise orthogonal to the design, so the
    fit is exact), and the boundary of Eq. 4 is its closed form.  Each case is
    chosen so that taking the minimum over all positions, or stopping one
    position before the break, gives a different number."""
    rng = np.random.default_rng(31)
    N, n_hist, f, lam, hf, k = 150, 64, 23.0, 1.8, 0.25, 2
    K = 2 + 2 * k
    d = synth.dates(4, N)
    valid = rng.random(N) > 0.25
    valid[0] = valid[n_hist] = True
    idx = np.nonzero(valid)[0]
    n = int((idx < n_hist).sum())
    P = idx.size - n
    h = max(1, min(int(math.floor(hf * n)), n))
    X = _design_np(d[idx], k, f)
    beta = np.array([0.5, 0.002, 0.1, -0.05, 0.03, 0.02])
    e = _orth_noise(X[:n], rng, 0.02)
    b = _boundary_np(lam, n, P)
    sgn = np.where(np.arange(P) % 2 == 0, 1.0, -1.0)
    if case == "min_at_break":
        mo = 0.5 * b * sgn
        j1, j2 = 20, 35
        mo[j1] = -(b[j1] + 0.004)               # first crossing (negative), margin 0.004
        mo[j2] = b[j2] - 0.001                  # closer, but after the break
        first, expect = j1, 0.004
    elif case == "min_before_break":
        mo = 0.4 * b * sgn
        j0, j1, j2 = 10, 30, 45
        mo[j0] = b[j0] - 0.0015                 # closest approach, no crossing
        mo[j1] = b[j1] + 0.01                   # first crossing
        mo[j2] = -(b[j2] + 0.0005)              # after the break
        first, expect = j1, 0.0015
    else:
        mo = 0.6 * b * sgn
        j3 = 40
        mo[j3] = -(b[j3] - 0.002)               # closest approach anywhere
        first, expect = -1, 0.002
    dist = np.abs(np.abs(mo) - b)
    upto = dist[: first + 1] if first >= 0 else dist
    assert abs(upto.min() - expect) < 1e-12
    # the slips named above give other values
    if case != "no_break":
        assert abs(dist.min() - expect) > 1e-4                 # minimum over all positions
    if case == "min_at_break":
        assert abs(dist[:first].min() - expect) > 1e-4         # stopping before the break
    r = _residuals_for_trace(e, mo, h, K)
    y = X @ beta + r
    Y = np.full((N, 1), np.nan)
    Y[idx, 0] = y
    o = oracle.monitor(d, Y, k=k, f=f, n_hist=n_hist, h_frac=hf, lam=lam, trace=True)
    assert o["status"][0] == 0 and o["n"][0] == n and o["h"][0] == h
    np.testing.assert_allclose(o["mo_trace"][0, :P], mo, rtol=1e-9, atol=1e-10)
    assert o["break_idx"][0] == (idx[n + first] if first >= 0 else -1)
    np.testing.assert_allclose(o["margin"][0], expect, rtol=1e-6)


def test_invariance_affine_in_model_space():
    """Adding a model-space vector X g leaves residuals (so MO, break, sigma)
    unchanged and shifts beta by g; scaling y by a > 0 scales beta and sigma
    by a and leaves MO unchanged."""
    w = synth.workload("c1", m=200)
    k, f = 3, w["f"]
    Y = w["Y"].astype(np.float64)
    X = _design_np(w["dates"], k, f)
    g = np.array([0.1, 0.0005, 0.05, -0.02, 0.01, 0.0, 0.02, -0.01])
    kw = dict(k=k, f=f, n_hist=w["n_hist"], h_frac=w["h_frac"], lam=w["lam"])
    o1 = oracle.monitor(w["dates"], Y, **kw, trace=True)
    o2 = oracle.monitor(w["dates"], Y + (X @ g)[:, None], **kw, trace=True)
    o3 = oracle.monitor(w["dates"], 3.0 * Y, **kw, trace=True)
    ok = o1["status"] == 0
    np.testing.assert_allclose(o2["beta"][:, ok], o1["beta"][:, ok] + g[:, None], atol=1e-10)
    np.testing.assert_allclose(o2["mo_trace"][ok], o1["mo_trace"][ok], atol=1e-8, equal_nan=True)
    np.testing.assert_allclose(o3["mo_trace"][ok], o1["mo_trace"][ok], atol=1e-9, equal_nan=True)
    np.testing.assert_allclose(o3["sigma"][ok], 3 * o1["sigma"][ok], rtol=1e-12)
    tie = o1["margin"] < 1e-6
    np.testing.assert_array_equal(o2["break_idx"][ok & ~tie], o1["break_idx"][ok & ~tie])


def test_edge_cases():
    """n_p <= K (INSUFFICIENT), no monitoring data (NO_MONITOR), all missing,
    bandwidth clamps to 1 and to n_p, and an exactly collinear history
    (SINGULAR: valid history dates one season apart make every harmonic
    column constant, i.e. a multiple of the intercept)."""
    f, N, n_hist = 23.0, 120, 60
    d = _dates_regular(N)
    rng = np.random.default_rng(0)
    Y = 0.5 + 0.03 * rng.standard_normal((N, 6))
    Y[8:n_hist, 0] = np.nan                      # 8 valid history obs <= K = 8
    Y[n_hist:, 1] = np.nan                       # no monitoring data
    Y[:, 2] = np.nan                             # all missing
    keep = np.zeros(N, bool)
    keep[np.arange(0, n_hist, 23)] = True        # t = 1, 24, 47: same phase
    keep[n_hist:] = True
    Y[~keep, 3] = np.nan
    o = oracle.monitor(d, Y, k=3, f=f, n_hist=n_hist, h_frac=0.25, lam=1.7)
    assert list(o["status"][:3]) == [1, 4, 1]
    assert o["n"][0] == 8 and o["Nv"][2] == 0
    assert np.isnan(o["beta"][:, 0]).all() and o["break_idx"][0] == -1
    assert np.isnan(o["mean_mosum"][1]) and o["break_idx"][1] == -1 and np.isfinite(o["sigma"][1])
    # column 3 has only 3 history obs -> INSUFFICIENT; give it more on the same phase
    Y2 = np.full((N, 1), np.nan)
    t_same = np.arange(0, N, 23)
    Y2[t_same, 0] = 0.5 + 0.01 * rng.standard_normal(t_same.size)
    o2 = oracle.monitor(d, Y2, k=1, f=f, n_hist=N - 10, h_frac=0.25, lam=1.7)
    assert o2["n"][0] > 4 and o2["status"][0] == 2
    # bandwidth clamps
    o3 = oracle.monitor(d, Y[:, 4:6], k=3, f=f, n_hist=n_hist, h_frac=1e-4, lam=1.7)
    assert (o3["h"] == 1).all()
    o4 = oracle.monitor(d, Y[:, 4:6], k=3, f=f, n_hist=n_hist, h_frac=1.0, lam=1.7)
    assert (o4["h"] == o4["n"]).all()


def test_mask_bits_and_int16_convention():
    """Explicit mask bits AND the in-band marker; int16 values are used as
    stored, -32768 is missing (the int16 scene is 1e4 x the float one up to
    rounding, so beta scales by 1e4 and MO is nearly unchanged)."""
    w = synth.workload("c1", m=96)
    wi = synth.workload("c3", m=96)
    N, m = w["N"], 96
    rng = np.random.default_rng(1)
    bits = rng.integers(0, 2**32, size=(N, 3), dtype=np.uint64).astype(np.uint32)
    kw = dict(k=3, f=w["f"], n_hist=w["n_hist"], h_frac=0.25, lam=w["lam"])
    o_mask = oracle.monitor(w["dates"], w["Y"], mask_bits=bits, **kw)
    p = np.arange(m)
    on = ((bits[:, p // 32] >> (p % 32).astype(np.uint32)) & 1).astype(bool)
    Ym = np.where(on, w["Y"], np.nan)
    o_ref = oracle.monitor(w["dates"], Ym, **kw)
    for key in ("break_idx", "status", "n", "Nv"):
        np.testing.assert_array_equal(o_mask[key], o_ref[key])
    np.testing.assert_array_equal(o_mask["beta"], o_ref["beta"])
    oi = oracle.monitor(wi["dates"], wi["Y"], **kw)
    of = oracle.monitor(w["dates"], w["Y"], **kw)
    ok = (oi["status"] == 0) & (of["status"] == 0)
    np.testing.assert_allclose(oi["beta"][0, ok], 1e4 * of["beta"][0, ok], rtol=1e-3)
    np.testing.assert_allclose(oi["mean_mosum"][ok], of["mean_mosum"][ok], atol=2e-2)


def test_lambda_matches_paper_value():
    """The paper's boundary 2.39 for alpha = 0.05, h/n = 0.5, N/n = 2
    (Section 4.3) from the simulated limiting process (weak pin)."""
    with open(os.path.join(GOLDEN, "paper_values.json")) as fh:
        g = json.load(fh)["critical_value_chile"]
    lam = oracle.critical_value(g["alpha"], g["h_over_n"], g["N_over_n"], G=800, reps=20000, seed=3)
    assert abs(lam - g["lambda"]) < g["tolerance"]


def test_lambda_monotone():
    """lambda grows with the horizon and as alpha shrinks."""
    a = oracle.critical_value(0.05, 0.25, 1.5, G=400, reps=8000, seed=1)
    b = oracle.critical_value(0.05, 0.25, 3.0, G=400, reps=8000, seed=1)
    c = oracle.critical_value(0.01, 0.25, 3.0, G=400, reps=8000, seed=1)
    assert a < b < c


@pytest.mark.parametrize("h", [0.25, 0.5])
def test_lambda_at_unit_horizon_is_half_normal(h):
    """At the horizon T = 1 the supremum runs over t = 1 alone, where
    log+ 1 = 1 and Z(1) = W(1) - W(1-h) - h W(1) = (1-h)(W(1) - W(1-h)) - h W(1-h)
    is normal with variance (1-h)^2 h + h^2 (1-h) = h(1-h).  So the simulated
    statistics follow the half-normal law of scale sqrt(h(1-h)) (Kolmogorov-
    Smirnov distance below its 1 % critical value) and lambda is
    sqrt(h(1-h)) z_{1-alpha/2} within four standard errors of an order statistic."""
    from statistics import NormalDist
    R, alpha = 40000, 0.05
    lam, st = oracle.critical_value(alpha, h, 1.0, G=200, reps=R, seed=7, return_stats=True)
    s = math.sqrt(h * (1.0 - h))
    x = np.sort(st)
    cdf = np.frompyfunc(lambda v: math.erf(v / (s * math.sqrt(2.0))), 1, 1)(x).astype(np.float64)
    D = max((np.arange(1, R + 1) / R - cdf).max(), (cdf - np.arange(R) / R).max())
    assert D < 1.63 / math.sqrt(R)
    nd = NormalDist()
    q = s * nd.inv_cdf(1.0 - alpha / 2.0)
    dens = 2.0 * nd.pdf(q / s) / s
    se = math.sqrt(alpha * (1.0 - alpha) / R) / dens
    assert abs(lam - q) < 4.0 * se


def test_lambda_table_consistent():
    """The stored workload critical values are what the oracle helper gives."""
    tab = synth.lambda_table()
    c2 = tab["workloads"]["c2"]
    lam = oracle.critical_value(c2["alpha"], c2["h"], c2["T"], G=400, reps=20000, seed=5)
    assert abs(lam - c2["lambda"]) < 0.04


def test_trend_extrapolation_inflates_null_crossings():
    """Stable series without any change: the model of Eq. 2 always carries a
    trend column, whose history estimate is extrapolated over the monitoring
    period; its error adds a drift of about sd(slope)*(t - t_hist_mean)*h to
    each window, so crossings grow with the horizon.  With a horizon of
    N/n = 1.25 the drift is small and the rate stays near alpha; with
    N/n = 2 it is several times alpha."""
    rng = np.random.default_rng(2)
    m, n = 3000, 200
    rates = []
    for N in (250, 400):
        d = _dates_regular(N)
        Y = 0.5 + 0.1 * np.sin(2 * np.pi * d / 23.0)[:, None] + 0.05 * rng.standard_normal((N, m))
        lam = oracle.critical_value(0.05, 0.25, N / n, G=800, reps=20000, seed=4)
        o = oracle.monitor(d, Y, k=1, f=23.0, n_hist=n, h_frac=0.25, lam=lam)
        rates.append((o["break_idx"] >= 0).mean())
    assert 0.01 < rates[0] < 0.12
    assert rates[1] > 2 * rates[0]


def test_max_mosum_definition():
    """max_mosum is the signed MO of largest magnitude over the monitoring
    positions: a downward step gives a negative value whose magnitude is the
    largest |MO| of the trace; DEGENERATE gives 0, too little history NaN."""
    w = synth.workload("c1", m=256)
    Y = w["Y"].copy()
    n = w["n_hist"]
    Y[n + 10:, 1] -= 0.5                                  # strong downward step
    Y[:, 2] = np.float32(0.25)                            # constant: DEGENERATE
    Y[6:n, 3] = np.nan                                    # too little history
    out = oracle.monitor(w["dates"], Y, k=3, f=23.0, n_hist=n, h_frac=0.25, lam=w["lam"], trace=True)
    mx = oracle.max_mosum(out)
    tr = out["mo_trace"]
    assert out["status"][1] == 0 and mx[1] < 0
    assert mx[1] == np.nanmin(tr[1]) and abs(mx[1]) == np.nanmax(np.abs(tr[1]))
    assert out["status"][2] == 3 and mx[2] == 0.0
    assert out["status"][3] == 1 and np.isnan(mx[3])
    ok = out["status"] == 0
    assert np.all(np.abs(mx[ok]) == np.nanmax(np.abs(tr[ok]), axis=1))


def test_shared_pseudo_inverse_on_complete_series():
    """Section 3, Eq. 8-11: without missing values every pixel shares the history design, so
    beta_all = M Y_h with one M = (X_h'X_h)^-1 X_h' (built here with numpy's pinv, independently
    of the oracle), the predictions are X beta_all and the residuals Y - X beta_all.  The oracle's
    per-pixel Householder fits, sigma-hat and MOSUM means must agree with that matrix algebra."""
    d, Y, _ = synth.scene(seed=9, m=64, N=120, n_hist=60, f=23.0, k_gen=2, intercept=0.5, slope=0.002,
                          coef_fixed=[0.2, 0.0, 0.0, 0.05], noise_sd=0.03, miss="none", break_frac=0.3,
                          step=(-0.3, -0.3), dtype="f32")
    n, h_frac, lam, k = 60, 0.25, 1.9, 2
    ref = oracle.monitor(d, Y, k=k, f=23.0, n_hist=n, h_frac=h_frac, lam=lam)
    X = _design_np(d, k, 23.0)
    Yd = Y.astype(np.float64)
    M = np.linalg.pinv(X[:n])                      # K x n, shared by every pixel
    B = M @ Yd[:n]                                 # K x m: beta_all = M Y_h
    R = Yd - X @ B                                 # residuals of every date
    K = X.shape[1]
    sig = np.sqrt((R[:n] ** 2).sum(axis=0) / (n - K))
    h = int(math.floor(h_frac * n))
    cs = np.vstack([np.zeros((1, Yd.shape[1])), np.cumsum(R, axis=0)])
    mo = np.array([(cs[j] - cs[j - h]) / (sig * math.sqrt(n)) for j in range(n + 1, Y.shape[0] + 1)])
    assert (ref["status"] == 0).all()
    np.testing.assert_allclose(ref["beta"], B, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(ref["sigma"], sig, rtol=1e-9)
    np.testing.assert_allclose(ref["mean_mosum"], mo.mean(axis=0), rtol=1e-9, atol=1e-12)
