"""Pins of the subsampled kernel RX oracle (oracle/krx.py), on the CPU.

Each pin comes from outside the oracle's own code path: RX of the background samples
(the linear-kernel special case), a closed form worked by hand, an eigendecomposition
identity, exact invariances of the Gaussian kernel, and planted mistakes that the pins
must reject.
"""
import math

import numpy as np
import pytest

from oracle import krx
from oracle import rx as orx


def _data(n=300, B=6, seed=0):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(B, B))
    return rng.normal(size=(n, B)) @ A.T + rng.normal(size=B) * 3.0


def test_linear_kernel_reduces_to_rx_of_the_background():
    """With k(x, y) = x^T y the centred Gram matrix is X~ X~^T (X~: the centred background,
    m x B) and k~_r = X~ r~, so by the push-through identity
        delta(r) = (m - 1) r~^T (C + lam I)^-1 C (C + lam I)^-1 r~,   C = X~^T X~,
    a B x B computation that shares nothing with the oracle's m x m Cholesky solves; as
    lam -> 0 it is RX (Eq. 1) of the background with the m - 1 sample covariance."""
    X = _data(400, 6)
    idx = np.arange(0, 400, 3)
    S = X[idx]
    m = S.shape[0]
    mu = orx.sample_mean(S)
    Xt = S - mu
    C = Xt.T @ Xt
    R = (X - mu).T
    for eps in (1e-3, 1e-6):
        bg = krx.krx_background(S, krx.LINEAR, eps=eps)
        d = krx.krx_scores(X, bg)
        lam = bg["lam"]
        assert abs(lam - eps * np.trace(C) / m) < 1e-9 * lam   # tr(K~) = tr(C)
        Z = np.linalg.solve(C + lam * np.eye(6), R)
        ref = (m - 1) * (Z * (C @ Z)).sum(axis=0)
        np.testing.assert_allclose(d, ref, rtol=1e-8)
    rx = orx.rx_scores(X, mu, orx.sample_covariance(S, mu))
    np.testing.assert_allclose(d, rx, rtol=1e-4)             # eps = 1e-6: the RX limit


def test_two_samples_one_band_closed_form():
    """m = 2, B = 1, s = (0, 1), c = 1: K~ = (1 - e^-1)/2 [[1, -1], [-1, 1]], its nonzero
    eigenvalue 1 - e^-1 along (1, -1)/sqrt 2, lam = eps (1 - e^-1) / 2, and for r = 1/4 with
    a = exp(-1/16), b = exp(-9/16): k~ = (a - b)/2 (1, -1), so
        delta = (a - b)^2 / (2 (1 - e^-1 + lam)^2)."""
    eps = 0.1
    bg = krx.krx_background(np.array([[0.0], [1.0]]), krx.RBF, c=1.0, eps=eps)
    d = krx.krx_scores(np.array([[0.25]]), bg)[0]
    a, b = math.exp(-1 / 16), math.exp(-9 / 16)
    lam = eps * (1 - math.exp(-1)) / 2
    assert abs(bg["lam"] - lam) < 1e-15
    assert abs(d - (a - b) ** 2 / (2 * (1 - math.exp(-1) + lam) ** 2)) < 1e-13


def test_default_width_is_the_mean_pairwise_distance():
    S = np.array([[0.0, 0.0], [3.0, 4.0], [6.0, 8.0]])
    # squared distances 25, 100, 25
    assert abs(krx.mean_pairwise_distance(S) - 50.0) < 1e-12
    assert abs(krx.krx_background(S)["c"] - 50.0) < 1e-12


def _in_sample_identity(bg):
    """(m - 1) sum_j l_j^2 / (l_j + lam)^2 over the eigenvalues of K~."""
    lj = np.linalg.eigvalsh(bg["Kc"])
    return (bg["m"] - 1) * float((lj ** 2 / (lj + bg["lam"]) ** 2).sum())


@pytest.mark.parametrize("eps", [1e-1, 1e-2, 1e-3])
def test_in_sample_scores_sum_to_the_spectral_identity(eps):
    """sum_i delta(s_i) = (m - 1) tr(K~ (K~ + lam I)^-2 K~) over the background samples,
    computed from an eigendecomposition instead of the Cholesky solves."""
    X = _data(200, 5, seed=1)
    bg = krx.krx_background(X[:64], krx.RBF, eps=eps)
    d = krx.krx_scores(X[:64], bg)
    assert abs(d.sum() - _in_sample_identity(bg)) <= 1e-9 * d.sum()


def test_gaussian_scores_invariant_under_translation_and_rotation():
    X = _data(150, 5, seed=2)
    idx = np.arange(0, 150, 2)
    d0, _ = krx.subsampled_krx(X, idx)
    q, _ = np.linalg.qr(np.random.default_rng(3).normal(size=(5, 5)))
    d1, _ = krx.subsampled_krx(X @ q.T + 7.5, idx)
    np.testing.assert_allclose(d1, d0, rtol=1e-9)


def test_calibration_offsets_cancel_and_gains_do_not():
    X = np.abs(_data(120, 4, seed=4)) * 100
    idx = np.arange(0, 120, 4)
    d0, _ = krx.subsampled_krx(X, idx)
    d_off, _ = krx.subsampled_krx(X, idx, offset=[5.0, 1.0, 2.0, 3.0])
    np.testing.assert_allclose(d_off, d0, rtol=1e-9)
    d_gain, _ = krx.subsampled_krx(X, idx, gain=[1.0, 2.0, 1.0, 0.5])
    assert np.abs(d_gain - d0).max() > 1e-3 * d0.max()


def test_implanted_anomalies_rank_high():
    """Pixels far from a two-cluster background score above every background pixel."""
    rng = np.random.default_rng(5)
    bgd = np.concatenate([rng.normal(0, 1, (300, 4)), rng.normal(6, 1, (300, 4))])
    anom = rng.normal(0, 1, (5, 4)) + np.array([3.0, -6.0, 3.0, 9.0])
    X = np.concatenate([bgd, anom])
    d, _ = krx.subsampled_krx(X, np.arange(0, 600, 3), eps=1e-2)
    assert d[600:].min() > np.percentile(d[:600], 99)


def test_rejects_repeated_or_out_of_range_indices():
    X = _data(20, 3)
    for idx in ([1, 1, 2], [0, 25], [-1, 3]):
        with pytest.raises(ValueError):
            krx.subsampled_krx(X, idx)


# ------------------------------------------------------------------ planted mistakes
@pytest.mark.parametrize("kind", ["width", "uncentred", "single_inverse", "m_not_m_minus_1"])
def test_planted_mistakes_are_rejected(kind, monkeypatch):
    """One plausible mistake planted in the oracle at a time: a kernel width twice the mean
    pairwise distance, an uncentred test vector, k~^T A^-1 k~ (one solve) instead of
    ||A^-1 k~||^2, and m instead of m - 1. The in-sample identity (eigenvalues of the
    correct K~) or the width pin must then fail."""
    X = _data(160, 5, seed=6)
    S = X[:48]
    ref = _in_sample_identity(krx.krx_background(S, krx.RBF, eps=1e-2))
    good = krx.krx_scores(S, krx.krx_background(S, krx.RBF, eps=1e-2)).sum()
    assert abs(good - ref) <= 1e-9 * ref
    if kind == "width":
        orig = krx.mean_pairwise_distance
        monkeypatch.setattr(krx, "mean_pairwise_distance", lambda S_: 2.0 * orig(S_))
    elif kind == "uncentred":
        monkeypatch.setattr(krx, "centered_test_vectors", lambda Kr, K: Kr)
    elif kind == "single_inverse":
        # stop after the forward solve: ||L^-1 k~||^2 = k~^T A^-1 k~
        monkeypatch.setattr(krx, "backward_substitution", lambda U, R: R)
    bg = krx.krx_background(S, krx.RBF, eps=1e-2)
    if kind == "m_not_m_minus_1":
        bg["m"] += 1
    bad = krx.krx_scores(S, bg).sum()
    assert abs(bad - ref) > 1e-6 * ref
    if kind == "width":
        assert abs(bg["c"] - krx.squared_distances(S, S)[np.triu_indices(48, 1)].mean()) > 1.0
