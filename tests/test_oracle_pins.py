"""Pins of the FP64 oracle against facts fixed outside it (CPU only).

Each test checks the oracle against something it does not compute itself:
exact rational arithmetic, hand-derived values, closed forms, exact
identities of the sample covariance, a distributional law, or LAPACK.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.stats

import oracle
from oracle import rx as orx
from tests._exact import exact_scores

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b, floor=1.0):
    return np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.maximum(np.abs(b), floor))


# ---------------------------------------------------------------- exact values
def test_hand_derived_golden_cases():
    """Hand-derived Eq. 1 values (tests/golden/hand_examples.json)."""
    cases = json.load(open(os.path.join(GOLDEN, "hand_examples.json")))["cases"]
    for c in cases:
        X = np.array(c["pixels"], dtype=np.float64)
        mu = oracle.sample_mean(X)
        S = oracle.sample_covariance(X, mu)
        d = oracle.rx_scores(np.array(c["scored"], dtype=np.float64), mu, S)
        np.testing.assert_allclose(d, c["expected"], rtol=1e-13, atol=1e-13, err_msg=c["name"])


@pytest.mark.parametrize("B,N,seed", [(1, 5, 0), (2, 6, 1), (3, 9, 2), (4, 8, 3), (5, 12, 4)])
def test_exact_rational_bruteforce(B, N, seed):
    """Oracle (Cholesky, FP64) vs exact Fractions (Gauss-Jordan) on tiny integer cubes."""
    rng = np.random.default_rng(seed)
    X = rng.integers(-20, 21, size=(N, B)).astype(np.float64)
    scored = np.vstack([X, rng.integers(-30, 31, size=(3, B))]).astype(np.float64)
    ex = np.array([float(v) for v in exact_scores(X.tolist(), scored.tolist())])
    mu = oracle.sample_mean(X)
    d = oracle.rx_scores(scored, mu, oracle.sample_covariance(X, mu))
    assert _rel(d, ex, floor=1e-12) < 1e-11


def test_exact_rational_bruteforce_noninteger():
    rng = np.random.default_rng(7)
    X = np.round(rng.normal(size=(10, 3)) * 64) / 64.0   # dyadic, exactly representable
    ex = np.array([float(v) for v in exact_scores(X.tolist(), X.tolist())])
    mu = oracle.sample_mean(X)
    d = oracle.rx_scores(X, mu, oracle.sample_covariance(X, mu))
    assert _rel(d, ex, floor=1e-12) < 1e-11


# ---------------------------------------------------------------- identities
@pytest.mark.parametrize("N,B", [(50, 3), (200, 10), (1000, 64)])
def test_in_sample_mean_identity(N, B):
    """sum_i delta_i = tr(Sigma^{-1} (N-1) Sigma) = B (N-1), so mean = B(N-1)/N."""
    rng = np.random.default_rng(N + B)
    A = rng.normal(size=(B, B))
    X = rng.normal(size=(N, B)) @ A + 5.0
    mu = oracle.sample_mean(X)
    d = oracle.rx_scores(X, mu, oracle.sample_covariance(X, mu))
    assert abs(d.mean() - B * (N - 1) / N) / (B * (N - 1) / N) < 1e-10
    # leverage bound: delta_i <= (N-1)^2 / N
    assert d.max() <= (N - 1) ** 2 / N * (1 + 1e-12)


def test_leverage_bound_attained_by_single_outlier():
    """With B = 1, a single far outlier approaches delta = (N-1)^2/N from below."""
    X = np.zeros((20, 1))
    X[-1] = 1e6
    X[:-1, 0] = np.linspace(-1, 1, 19)
    mu = oracle.sample_mean(X)
    d = oracle.rx_scores(X, mu, oracle.sample_covariance(X, mu))
    bound = 19 ** 2 / 20
    assert d[-1] <= bound and d[-1] > bound * (1 - 1e-6)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_affine_invariance(seed):
    """delta unchanged under x -> A x + b for invertible A (Sec. 2.1: linear maps do not change RX)."""
    rng = np.random.default_rng(seed)
    N, B = 300, 12
    X = rng.normal(size=(N, B)) @ rng.normal(size=(B, B))
    A = rng.normal(size=(B, B)) + 3 * np.eye(B)
    b = rng.normal(size=B) * 10
    Y = X @ A.T + b
    def scores(Z):
        mu = oracle.sample_mean(Z)
        return oracle.rx_scores(Z, mu, oracle.sample_covariance(Z, mu))
    assert _rel(scores(Y), scores(X)) < 1e-9
    # per-band gain / offset through calibrate(), and a band permutation
    gain, off = rng.uniform(0.1, 5.0, B), rng.uniform(-50, 50, B)
    assert _rel(scores(oracle.calibrate(X, gain, off)), scores(X)) < 1e-9
    perm = rng.permutation(B)
    assert _rel(scores(X[:, perm]), scores(X)) < 1e-9


# ---------------------------------------------------------------- closed forms
def test_closed_form_one_band():
    """B = 1: delta = (s - mean)^2 / s^2 with s^2 the N-1 sample variance."""
    rng = np.random.default_rng(11)
    x = rng.normal(3.0, 2.0, size=37)
    m = x.sum() / x.size
    var = ((x - m) ** 2).sum() / (x.size - 1)
    d = oracle.rx_scores(x[:, None], oracle.sample_mean(x[:, None]),
                         oracle.sample_covariance(x[:, None], oracle.sample_mean(x[:, None])))
    assert _rel(d, (x - m) ** 2 / var, floor=1e-12) < 1e-12


def test_closed_form_two_bands():
    """B = 2: explicit inverse [[c, -b], [-b, a]] / (ac - b^2)."""
    rng = np.random.default_rng(12)
    X = rng.normal(size=(41, 2)) @ np.array([[2.0, 0.7], [0.0, 0.5]])
    mu = X.mean(0)
    D = X - mu
    a, b, c = (D[:, 0] ** 2).sum() / 40, (D[:, 0] * D[:, 1]).sum() / 40, (D[:, 1] ** 2).sum() / 40
    ref = (c * D[:, 0] ** 2 - 2 * b * D[:, 0] * D[:, 1] + a * D[:, 1] ** 2) / (a * c - b * b)
    d = oracle.rx_scores(X, oracle.sample_mean(X), oracle.sample_covariance(X, oracle.sample_mean(X)))
    assert _rel(d, ref, floor=1e-12) < 1e-12


def test_zero_at_mean():
    """Sec. 3.3: the score is zero for a pixel equal to the mean."""
    rng = np.random.default_rng(13)
    X = rng.normal(size=(100, 7)) @ rng.normal(size=(7, 7))
    mu = oracle.sample_mean(X)
    d = oracle.rx_scores(mu[None, :], mu, oracle.sample_covariance(X, mu))
    assert abs(d[0]) < 1e-20


def test_inverse_variance_scaling():
    """Sec. 3.3: for a fixed offset the score falls inversely with the variance of that band."""
    rng = np.random.default_rng(14)
    X = rng.normal(size=(500, 3))
    mu = oracle.sample_mean(X)
    S = oracle.sample_covariance(X, mu)
    e = np.zeros(3)
    e[0] = 1.0
    d1 = oracle.rx_scores((mu + e)[None], mu, S)[0]
    X2 = X.copy()
    X2[:, 0] *= 4.0     # variance x16 along band 0, same offset
    mu2 = oracle.sample_mean(X2)
    d2 = oracle.rx_scores((mu2 + e)[None], mu2, oracle.sample_covariance(X2, mu2))[0]
    assert abs(d1 / d2 - 16.0) < 1e-9


def test_out_of_sample_scores_follow_hotelling_t2():
    """Independent x ~ N(mu, Sigma) scored against N samples: N(N-B)/(B(N+1)(N-1)) delta ~ F(B, N-B)."""
    rng = np.random.default_rng(15)
    N, B, trials = 30, 4, 3000
    vals = np.empty(trials)
    A = rng.normal(size=(B, B)) + 2 * np.eye(B)
    for k in range(trials):
        Z = rng.normal(size=(N + 1, B)) @ A.T + 3.0
        mu = oracle.sample_mean(Z[:N])
        vals[k] = oracle.rx_scores(Z[N:], mu, oracle.sample_covariance(Z[:N], mu))[0]
    f = vals * N * (N - B) / (B * (N + 1) * (N - 1))
    assert scipy.stats.kstest(f, scipy.stats.f(B, N - B).cdf).pvalue > 1e-3
    expect = B * (N - 1) * (N + 1) / (N * (N - B - 2))
    assert abs(vals.mean() - expect) / expect < 0.06


# ---------------------------------------------------------------- library routines
@pytest.mark.parametrize("B", [1, 2, 17, 64, 130])
def test_cholesky_and_substitution_vs_lapack(B):
    rng = np.random.default_rng(B)
    A = rng.normal(size=(B, 3 * B + 5))
    S = A @ A.T / (3 * B + 4)
    L = oracle.cholesky_lower(S)
    np.testing.assert_allclose(L, np.linalg.cholesky(S), rtol=1e-10, atol=1e-12)
    assert np.linalg.norm(L @ L.T - S) / np.linalg.norm(S) < 1e-13
    R = rng.normal(size=(B, 9))
    np.testing.assert_allclose(oracle.forward_substitution(L, R),
                               scipy.linalg.solve_triangular(L, R, lower=True), rtol=1e-9, atol=1e-12)


def test_not_positive_definite_detected():
    X = np.random.default_rng(0).normal(size=(40, 5))
    X[:, 2] = 7.0                       # constant band -> zero variance
    mu = oracle.sample_mean(X)
    with pytest.raises(oracle.NotPositiveDefinite):
        oracle.cholesky_lower(oracle.sample_covariance(X, mu))
    lines = X.reshape(8, 5, 5)
    d, st = orx.stream_rx_line(lines, 7, oracle.EXCLUSIVE)
    assert st == orx.NOT_PD and np.isnan(d).all()


# ---------------------------------------------------------------- thresholds
def test_threshold_strict_and_relative():
    d = np.array([0.0, 1.0, 2.0, 4.0, np.nan])
    assert oracle.threshold_mask(d, 2.0, oracle.ABS).tolist() == [False, False, False, True, False]
    # REL: delta / max > tau, max = 4
    assert oracle.threshold_mask(d, 0.5, oracle.REL).tolist() == [False, False, False, True, False]
    assert oracle.threshold_mask(d, 0.49, oracle.REL).tolist() == [False, False, True, True, False]


# ---------------------------------------------------------------- streamed forms
def _small_stream(T=12, W=6, B=4, seed=3):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 4096, size=(T, W, B)).astype(np.uint16)


def test_stream_windows_and_warmup():
    lines = _small_stream()
    T, W, B = lines.shape
    d, st = oracle.stream_rx(lines, oracle.EXCLUSIVE)
    # EXCLUSIVE: line 0 has no statistics, line 1 has W = 6 >= B+1 = 5 pixels
    assert st[0] == orx.NOT_READY and np.isnan(d[0]).all()
    assert (st[1:] == orx.OK).all()
    # warm-up threshold in pixels
    d2, st2 = oracle.stream_rx(lines, oracle.EXCLUSIVE, warmup_pixels=20)
    assert (st2[:4] == orx.NOT_READY).all() and (st2[4:] == orx.OK).all()
    np.testing.assert_array_equal(d2[4:], d[4:])


def test_exclusive_equals_global_stats_of_prior_lines():
    lines = _small_stream()
    t = 7
    d, _ = orx.stream_rx_line(lines, t, oracle.EXCLUSIVE)
    X = lines[:t].reshape(-1, lines.shape[2]).astype(np.float64)
    mu = oracle.sample_mean(X)
    ref = oracle.rx_scores(lines[t].astype(np.float64), mu, oracle.sample_covariance(X, mu))
    assert _rel(d, ref) < 1e-12


def test_inclusive_last_line_equals_cube_mode():
    lines = _small_stream(T=10)
    dc, _ = oracle.global_rx(lines)
    di, st = orx.stream_rx_line(lines, 9, oracle.INCLUSIVE)
    assert st == orx.OK and _rel(di, dc[9]) < 1e-12
    # with resets every 5 lines, line 9 closes the second cube
    dcube, _ = oracle.stream_rx(lines, oracle.CUBE, cube_lines=5)
    dc2, _ = oracle.global_rx(lines[5:10])
    assert _rel(dcube[5:10], dc2) < 1e-12
    di2, _ = orx.stream_rx_line(lines, 9, oracle.INCLUSIVE, cube_lines=5)
    assert _rel(di2, dc2[4]) < 1e-12


def test_leave_one_out_identity_links_exclusive_and_inclusive():
    """One pixel per line: the EXCLUSIVE score is a closed function of the INCLUSIVE one.

    With n pixels in the inclusive set, q = D_in / (n-1), c = n/(n-1):
    D_ex = c^2 (n-2) q / (1 - c q)   (Sherman-Morrison on the N-1 covariance).
    """
    rng = np.random.default_rng(21)
    T, B = 40, 3
    lines = (rng.normal(size=(T, 1, B)) @ rng.normal(size=(B, B)) + 1.0)
    for t in (B + 3, 20, 39):
        de, _ = orx.stream_rx_line(lines, t, oracle.EXCLUSIVE)
        di, _ = orx.stream_rx_line(lines, t, oracle.INCLUSIVE)
        n = t + 1
        q, c = di[0] / (n - 1), n / (n - 1)
        pred = c * c * (n - 2) * q / (1 - c * q)
        assert abs(de[0] - pred) / pred < 1e-9


def test_chunking_does_not_change_statistics():
    lines = _small_stream(T=9).astype(np.float64)
    mu1, S1, n1 = orx._stats_over_lines(lines, 0, 9, None, None, chunk=1)
    mu2, S2, n2 = orx._stats_over_lines(lines, 0, 9, None, None, chunk=64)
    assert n1 == n2 == 54
    assert _rel(S1, S2) < 1e-13 and _rel(mu1, mu2) < 1e-13


# ---------------------------------------------------------------- implanted anomalies
def _auc(pos, neg):
    allv = np.concatenate([pos, neg])
    ranks = scipy.stats.rankdata(allv)
    return (ranks[:pos.size].sum() - pos.size * (pos.size + 1) / 2) / (pos.size * neg.size)


def test_implanted_anomalies_rank_above_background():
    from gen import config1_cube
    cube, anom, _ = config1_cube()
    d, dn = oracle.global_rx(cube)
    assert anom.sum() == 80
    assert np.median(d[anom]) > np.percentile(d[~anom], 99)
    assert _auc(d[anom], d[~anom]) >= 0.99
    assert abs(dn.max() - 1.0) < 1e-15
    assert abs(d.mean() - 64 * (cube[..., 0].size - 1) / cube[..., 0].size) < 1e-8


def test_pushbroom_anomalies_rank_above_background():
    from gen import PushbroomScene
    sc = PushbroomScene(96, 24, seed=5)
    lines = sc.lines(0, 192)
    m = sc.anomaly_mask(0, 192)
    # the last 64 lines scored against the statistics of the first 128
    X = oracle.calibrate(lines[:128].reshape(-1, 24), sc.gain, sc.offset)
    mu = oracle.sample_mean(X)
    S = oracle.sample_covariance(X, mu)
    dd = oracle.rx_scores(oracle.calibrate(lines[128:].reshape(-1, 24), sc.gain, sc.offset), mu, S)
    mm = m[128:].reshape(-1)
    assert mm.sum() > 0
    assert _auc(dd[mm], dd[~mm]) > 0.99
    assert np.median(dd[mm]) > np.percentile(dd[~mm], 99)


# ------------------------------------------------------------------ transmit encoding (Sec. 3.4)
def _binary16_value(c):
    """Value of a binary16 bit pattern, decoded field by field (sign, exponent, mantissa)."""
    c = int(c)
    sign = -1.0 if c >> 15 else 1.0
    e, m = (c >> 10) & 31, c & 1023
    if e == 0:
        return sign * m / 1024.0 * 2.0 ** -14
    if e == 31:
        return sign * (math.inf if m == 0 else math.nan)
    return sign * (1.0 + m / 1024.0) * 2.0 ** (e - 15)


def test_transmit_encoding_hand_values():
    # binary16: 1.0 = 0x3C00, 0.5 = 0x3800, 1/3 -> exponent -2, mantissa 341 -> 0x3555
    codes, dmax = oracle.encode_tx([0.0, 1.0, 4.0])
    assert dmax == 4.0 and list(codes) == [0x0000, 0x3800, 0x3C00]
    codes, _ = oracle.encode_tx([9.0, 1.0])
    assert list(codes) == [0x3C00, 0x3555]
    codes, dmax = oracle.encode_tx([float("nan"), 2.0, float("inf")])
    assert dmax == 2.0 and codes[0] == 0x7E00 and codes[1] == 0x3C00 and codes[2] == 0x7C00
    codes, dmax = oracle.encode_tx([0.0, 0.0, float("nan")])  # no positive maximum: zeros stay zero
    assert dmax == 0.0 and list(codes[:2]) == [0, 0] and codes[2] == 0x7E00


def test_transmit_encoding_rounds_to_nearest_and_is_monotone():
    rng = np.random.default_rng(5)
    s = np.concatenate([rng.gamma(0.7, 30.0, 4000), [0.0, 1e-30, 7e3]]).astype(np.float32)
    codes, dmax = oracle.encode_tx(s)
    r64 = np.sqrt(s.astype(np.float64) / dmax)
    for c, r in zip(codes[:600], r64[:600]):
        v = _binary16_value(c)
        # the nearest binary16 value to the (FP32) ratio: no neighbour is closer by more than
        # the FP32 rounding of the ratio itself
        tol = 2.0 ** -23 * max(r, 2.0 ** -14)
        assert abs(v - r) <= abs(_binary16_value(c + 1) - r) + tol
        if c > 0:
            assert abs(v - r) <= abs(_binary16_value(c - 1) - r) + tol
    order = np.argsort(s, kind="stable")
    assert (np.diff(codes[order].astype(np.int64)) >= 0).all()
    assert codes[np.argmax(s)] == 0x3C00


# ------------------------------------------------------------------ front end (Sec. 3.2)
def test_frontend_band_discard_and_binning():
    raw = np.arange(2 * 3 * 12, dtype=np.uint16).reshape(2, 3, 12)
    out = oracle.frontend(raw, first=1, bin_=4, bands=2)
    # pixel (0, 0): raw bands 0..11 hold 0..11; kept 1..8, binned (1+2+3+4, 5+6+7+8)
    assert out.shape == (2, 3, 2) and list(out[0, 0]) == [10, 26]
    assert (out.sum(axis=-1) == raw[..., 1:9].astype(np.int64).sum(axis=-1)).all()
    assert (oracle.frontend(raw, 0, 1, 12) == raw).all()
    with pytest.raises(ValueError):
        oracle.frontend(raw, 5, 4, 2)


# ------------------------------------------------------------------ factorisation cadence (extension)
def test_cadence_window_and_scores():
    rng = np.random.default_rng(12)
    T, W, B = 11, 6, 3
    lines = rng.normal(size=(T, W, B)) @ np.diag([1.0, 2.0, 0.5]) + 10.0
    k = 3
    d1, s1 = orx.stream_rx(lines, oracle.EXCLUSIVE)
    dk, sk = orx.stream_rx(lines, oracle.EXCLUSIVE, every=k)
    for t in range(T):
        snap = k * (t // k)              # the last multiple of k lines: the statistics of lines [0, snap)
        if snap * W < B + 1:
            assert sk[t] == orx.NOT_READY and np.isnan(dk[t]).all()
            continue
        X = lines[:snap].reshape(-1, B)
        mu = X.mean(axis=0)
        D = X - mu
        Sigma = D.T @ D / (X.shape[0] - 1)
        ref = np.einsum("pi,ij,pj->p", lines[t] - mu, np.linalg.inv(Sigma), lines[t] - mu)
        np.testing.assert_allclose(dk[t], ref, rtol=1e-10)
        if t % k == 0:                   # at a snapshot line the cadence changes nothing
            np.testing.assert_array_equal(dk[t], d1[t])
    with pytest.raises(ValueError):
        orx.statistics_lines(4, oracle.INCLUSIVE, 0, 10, every=2)


# ------------------------------------------------------------------ per-line gain correction (Sec. 3.2)
def test_gain_correct_hand_values():
    v = np.array([[[2.0, 4.0]], [[6.0, 8.0]], [[3.0, 9.0]]])        # 3 lines x 1 pixel x 2 bands
    u = oracle.gain_correct(v, [2.0, 4.0, 0.5])
    np.testing.assert_array_equal(u[:, 0, :], [[1.0, 2.0], [1.5, 2.0], [6.0, 18.0]])
    for bad in ([1.0, 0.0, 1.0], [1.0, -2.0, 1.0], [1.0, np.nan, 1.0], [1.0, 1.0]):
        with pytest.raises(ValueError):
            oracle.gain_correct(v, bad)


def _gain_scene(seed=21, T=14, W=9, B=3):
    rng = np.random.default_rng(seed)
    R = rng.integers(40, 400, size=(T, W, B)).astype(np.float64)
    g = rng.choice([0.5, 1.0, 2.0, 4.0], size=T)          # powers of two: g_t R_t is exact
    return R, g, R * g[:, None, None]


@pytest.mark.parametrize("mode", [oracle.EXCLUSIVE, oracle.INCLUSIVE])
def test_line_gain_recovers_the_scene(mode):
    """A line recorded at gain g_t holds g_t times the scene; after the correction the
    scores are those of the scene itself, line by line and with every line's statistics."""
    R, g, DN = _gain_scene()
    d_ref, s_ref = orx.stream_rx(R, mode)
    d_g, s_g = orx.stream_rx(DN, mode, line_gain=g)
    np.testing.assert_array_equal(s_g, s_ref)
    ok = s_ref == orx.OK
    assert ok.sum() >= 10
    np.testing.assert_allclose(d_g[ok], d_ref[ok], rtol=1e-11)
    # without the correction the varying gain changes the scores
    d_raw, _ = orx.stream_rx(DN, mode)
    assert np.max(np.abs(d_raw[ok] - d_ref[ok]) / d_ref[ok]) > 1e-2


def test_line_gain_precedes_the_band_calibration():
    """Sec. 3.2 corrects the gain first and calibrates after: a per-band affine map after
    the correction leaves the scores unchanged; the offset subtracted before the division
    (the other order) does not."""
    R, g, DN = _gain_scene(seed=22)
    off = np.array([30.0, 55.0, 17.0])
    bg = np.array([0.5, 2.0, 1.25])
    d0, s0 = orx.stream_rx(DN, oracle.EXCLUSIVE, line_gain=g)
    d1, s1 = orx.stream_rx(DN, oracle.EXCLUSIVE, line_gain=g, gain=bg, offset=off)
    ok = s0 == orx.OK
    np.testing.assert_array_equal(s0, s1)
    np.testing.assert_allclose(d1[ok], d0[ok], rtol=1e-9)
    d2, _ = orx.stream_rx(DN - off, oracle.EXCLUSIVE, line_gain=g)
    assert np.max(np.abs(d2[ok] - d0[ok]) / d0[ok]) > 1e-3


# ------------------------------------------------------------------ exponential forgetting (extension)
@pytest.mark.parametrize("mode", [oracle.EXCLUSIVE, oracle.INCLUSIVE])
def test_forgetting_equals_replicated_pixels_exactly(mode):
    """With lam = 1/2 the weights of the window's lines are 2^-age; scaling them by 2^K makes
    them integers, i.e. line tau's pixels repeated 2^(K - age) times. The weighted mean is
    that of the repeated set, and the weighted N-1 covariance is the repeated set's times
    (N' - 1) / (N' - 2^K) (N' repeated pixels): checked against exact rational arithmetic."""
    from fractions import Fraction
    rng = np.random.default_rng(17)
    T, W, B = 6, 3, 2
    lines = rng.integers(-9, 10, size=(T, W, B)).astype(np.float64)
    d, st = orx.stream_rx(lines, mode, forget=0.5)
    checked = 0
    for t in range(T):
        a, b = orx.statistics_lines(t, mode, 0, T)
        K = b - 1 - a                                   # the oldest line's age
        rows = []
        for tau in range(a, b):
            rows += [list(p) for p in lines[tau]] * (2 ** (K - (b - 1 - tau)))
        n_w = Fraction(W) * sum(Fraction(1, 2 ** (b - 1 - tau)) for tau in range(a, b))
        if n_w < B + 1:
            assert st[t] == orx.NOT_READY and np.isnan(d[t]).all()
            continue
        ex = exact_scores(rows, lines[t].tolist())
        n_rep = len(rows)
        f = Fraction(n_rep - 2 ** K, n_rep - 1)
        ref = np.array([float(v * f) for v in ex])
        np.testing.assert_allclose(d[t], ref, rtol=1e-11)
        checked += 1
    assert checked >= 3


def test_forgetting_limits():
    rng = np.random.default_rng(18)
    lines = rng.normal(size=(9, 5, 3)) + 4.0
    d1, s1 = orx.stream_rx(lines, oracle.EXCLUSIVE)
    df, sf = orx.stream_rx(lines, oracle.EXCLUSIVE, forget=1.0)
    np.testing.assert_array_equal(s1, sf)
    np.testing.assert_array_equal(d1, df)
    # N saturates at W / (1 - lam) = 4 = B + 1 from below: no line is ever ready
    _, s = orx.stream_rx(rng.normal(size=(30, 2, 3)), oracle.EXCLUSIVE, forget=0.5)
    assert (s == orx.NOT_READY).all()
    np.testing.assert_allclose(oracle.forget_weights(3, 7, 0.5), [0.125, 0.25, 0.5, 1.0])
    for bad in (dict(forget=0.0), dict(forget=1.5), dict(forget=0.9, every=2)):
        with pytest.raises(ValueError):
            orx.stream_rx(lines, oracle.EXCLUSIVE, **bad)
    with pytest.raises(ValueError):
        orx.stream_rx(lines, oracle.CUBE, cube_lines=9, forget=0.9)
