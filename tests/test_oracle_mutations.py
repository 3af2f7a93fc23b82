"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin catches each.

A pin that passes a broken oracle pins nothing; each mutant below must be
rejected by at least one of the independent checks.
"""
import numpy as np
import pytest

import oracle
from oracle import rx as orx
from tests._exact import exact_scores


def _cov_biased(X, mu):                       # denominator N instead of N-1
    D = np.asarray(X, dtype=np.float64) - mu
    return (D.T @ D) / X.shape[0]


def _cov_no_centering(X, mu):                 # dropped mean subtraction
    X = np.asarray(X, dtype=np.float64)
    return (X.T @ X) / (X.shape[0] - 1)


def _fsub_transposed(L, R):                   # solves with L^T instead of L
    return np.linalg.solve(L.T, R)


def _chol_sign(S):                            # wrong sign in the pivot update
    S = np.asarray(S, dtype=np.float64)
    n = S.shape[0]
    L = np.zeros_like(S)
    for j in range(n):
        piv = S[j, j] + L[j, :j] @ L[j, :j]
        L[j, j] = np.sqrt(piv)
        L[j + 1:, j] = (S[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def _mean_off_by_one(X):                      # divides by N-1
    X = np.asarray(X, dtype=np.float64)
    return X.sum(axis=0) / (X.shape[0] - 1)


def _checks_fail():
    """Return True if at least one independent pin rejects the current oracle."""
    rng = np.random.default_rng(5)
    X = rng.integers(-20, 21, size=(9, 3)).astype(np.float64)
    ex = np.array([float(v) for v in exact_scores(X.tolist(), X.tolist())])
    try:
        mu = oracle.sample_mean(X)
        d = oracle.rx_scores(X, mu, oracle.sample_covariance(X, mu))
    except Exception:
        return True
    if not np.all(np.isfinite(d)):
        return True
    if np.max(np.abs(d - ex) / np.maximum(ex, 1e-12)) > 1e-11:
        return True
    N, B = X.shape
    return abs(d.mean() - B * (N - 1) / N) > 1e-10


@pytest.mark.parametrize("target,mutant", [
    ("sample_covariance", _cov_biased),
    ("sample_covariance", _cov_no_centering),
    ("forward_substitution", _fsub_transposed),
    ("cholesky_lower", _chol_sign),
    ("sample_mean", _mean_off_by_one),
])
def test_pins_reject_mutant(monkeypatch, target, mutant):
    assert not _checks_fail(), "pins must accept the unmodified oracle"
    monkeypatch.setattr(orx, target, mutant)
    monkeypatch.setattr(oracle, target, mutant)
    assert _checks_fail(), f"mutant {mutant.__name__} of {target} was not caught"


def _encode_no_sqrt(scores):                  # drops the square root
    s = np.asarray(scores, dtype=np.float32)
    dmax = np.float32(s[np.isfinite(s)].max())
    return (s / dmax).astype(np.float16).view(np.uint16), float(dmax)


def _encode_by_sum(scores):                   # normalises by the sum instead of the maximum
    s = np.asarray(scores, dtype=np.float32)
    tot = np.float32(s[np.isfinite(s)].sum())
    return np.sqrt(s / tot).astype(np.float16).view(np.uint16), float(tot)


def _frontend_shifted(raw, first, bin_, bands):  # bins start one band late
    raw = np.asarray(raw)[..., first + 1:first + 1 + bin_ * bands].astype(np.int64)
    return raw.reshape(raw.shape[:-1] + (bands, bin_)).sum(axis=-1)


@pytest.mark.parametrize("target,mutant", [("encode_tx", _encode_no_sqrt), ("encode_tx", _encode_by_sum),
                                           ("frontend", _frontend_shifted)])
def test_encoding_and_front_end_pins_reject_mutant(monkeypatch, target, mutant):
    import tests.test_oracle_pins as pins
    checks = [pins.test_transmit_encoding_hand_values, pins.test_frontend_band_discard_and_binning]

    def fails():
        for c in checks:
            try:
                c()
            except AssertionError:
                return True
        return False

    assert not fails(), "pins must accept the unmodified oracle"
    monkeypatch.setattr(orx, target, mutant)
    monkeypatch.setattr(oracle, target, mutant)
    assert fails(), f"mutant {mutant.__name__} of {target} was not caught"


def _gain_multiplied(v, line_gain):             # multiplies by the gain instead of dividing
    v = np.asarray(v, dtype=np.float64)
    return v * np.asarray(line_gain, dtype=np.float64).reshape((-1,) + (1,) * (v.ndim - 1))


def _gain_of_next_line(v, line_gain):           # line t corrected with the gain of line t + 1
    v = np.asarray(v, dtype=np.float64)
    g = np.roll(np.asarray(line_gain, dtype=np.float64).reshape(-1), -1)
    return v / g.reshape((-1,) + (1,) * (v.ndim - 1))


@pytest.mark.parametrize("mutant", [_gain_multiplied, _gain_of_next_line])
def test_gain_correction_pins_reject_mutant(monkeypatch, mutant):
    import tests.test_oracle_pins as pins
    checks = [pins.test_gain_correct_hand_values,
              lambda: pins.test_line_gain_recovers_the_scene(oracle.EXCLUSIVE)]

    def fails():
        for c in checks:
            try:
                c()
            except AssertionError:
                return True
        return False

    assert not fails(), "pins must accept the unmodified oracle"
    monkeypatch.setattr(orx, "gain_correct", mutant)
    monkeypatch.setattr(oracle, "gain_correct", mutant)
    assert fails(), f"mutant {mutant.__name__} of gain_correct was not caught"


def _weights_age_off_by_one(a, b, lam):       # the newest line already decayed once
    return np.asarray([float(lam) ** (b - tau) for tau in range(a, b)], dtype=np.float64)


def _weights_reversed(a, b, lam):             # the oldest line weighs 1
    return np.asarray([float(lam) ** (tau - a) for tau in range(a, b)], dtype=np.float64)


@pytest.mark.parametrize("mutant", [_weights_age_off_by_one, _weights_reversed])
def test_forgetting_pin_rejects_mutant(monkeypatch, mutant):
    import tests.test_oracle_pins as pins

    def fails():
        try:
            pins.test_forgetting_equals_replicated_pixels_exactly(oracle.EXCLUSIVE)
        except AssertionError:
            return True
        return False

    assert not fails(), "pins must accept the unmodified oracle"
    monkeypatch.setattr(orx, "forget_weights", mutant)
    monkeypatch.setattr(oracle, "forget_weights", mutant)
    assert fails(), f"mutant {mutant.__name__} of forget_weights was not caught"
