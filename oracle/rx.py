"""FP64 oracle of the RX detector (test infrastructure; never called by the library).

What it computes, and where the paper says so:

* Calibration, Sec. 3.2 ("Data Acquisition"): raw values are gain-corrected and
  radiometrically calibrated before detection. Reading: a per-band affine map
  x_b = (v_b - offset_b) * gain_b.
* Statistics, Sec. 3.3 ("Detection Algorithm"): each band is a variable and each
  pixel a sample; the mean is the per-band average and the covariance uses
  "standard statistical methods". Reading: the unbiased sample covariance with
  denominator N-1, computed two-pass (mean first, then the centred sum).
* Score, Sec. 3.3, Eq. 1: delta = (s - mu)^T Sigma^{-1} (s - mu), evaluated by
  the textbook Cholesky factorisation Sigma = L L^T, forward substitution
  z = L^{-1}(s - mu) and delta = z^T z.
* Normalisation and threshold, Sec. 3.3 (last paragraph): scores are divided by
  the cube maximum so the highest is 1; a pixel is anomalous when its score is
  above a configurable value. Reading: strict ">" on delta (ABS) or on
  delta / delta_max (REL).
* Statistics window. Global RX uses every pixel of the 1000-line cube,
  including the scored pixel (Sec. 3.3, first paragraph). A line-based detector
  is proposed in Sec. 6.1. Readings for the streamed forms: EXCLUSIVE scores
  line t against lines [r, t) and INCLUSIVE against [r, t], where r is the last
  reset (every ``cube_lines`` lines, or never when it is 0). A line whose
  statistics hold fewer than max(B+1, warmup_pixels) pixels is not ready
  (NaN score).
* Factorisation cadence (an extension; the paper does not define one): with a
  cadence of k lines, EXCLUSIVE statistics are taken only every k lines after the
  reset, and line t is scored against the last snapshot, [r, r + k floor((t-r)/k)).

* Transmit encoding, Sec. 3.4 ("Data Transmission"): each score is sent as an
  IEEE-754 half-precision value of its square root, normalised to the cube's
  maximum; the scores themselves are computed in single precision. Reading: code =
  binary16(sqrt(delta / delta_max)) with the division and the square root in FP32
  and round-to-nearest-even to binary16, delta_max the largest finite score of the
  block being sent; NaN scores stay NaN.
* Front end, Sec. 3.2 ("Data Acquisition"): the out-of-specification bands are
  discarded and four consecutive bands are summed into one. Reading: keep raw bands
  [first, first + bin * B) and sum groups of ``bin`` consecutive bands (integers, exact).
* Exponential forgetting (an extension; the paper does not define one, and names drift
  and cloud shadow as open problems for the statistics in Sec. 6.1). Reading: with a
  factor lam in (0, 1], every pixel of a window line tau counts with frequency weight
  lam^(b - 1 - tau), b the end of the window (the newest line weighs 1); N = sum of the
  weights, mu the weighted mean, Sigma = sum_p w_p (x_p - mu)(x_p - mu)^T / (N - 1), and a
  line is scored once N >= max(B + 1, warmup_pixels). lam = 1 is the unweighted window.
* Per-line gain correction, Sec. 3.2 ("Data Acquisition"): the imager's gain is changed
  for every line to avoid saturation, and the data is corrected for the varying gain
  before the radiometric calibration. Reading: one positive scalar g_t per line, every
  value of line t divided by it (u = v / g_t), then the per-band calibration above.

Pins (tests/test_oracle_*.py): exact rational brute force on tiny inputs, the
in-sample identity mean(delta) = B (N-1)/N, invariance under invertible affine
band maps, closed forms for B = 1 and B = 2, delta(mu) = 0, the Hotelling T^2
expectation for out-of-sample scores, the leave-one-out identity linking
EXCLUSIVE and INCLUSIVE scores, LAPACK's Cholesky and triangular solve, and
ranking of implanted anomalies.
"""
from __future__ import annotations

import math
from typing import Callable, Union

import numpy as np

EXCLUSIVE, INCLUSIVE, CUBE = "exclusive", "inclusive", "cube"
ABS, REL = "abs", "rel"

# per-line status codes returned by stream_rx
OK, NOT_READY, NOT_PD = 0, 1, 2


class NotPositiveDefinite(ArithmeticError):
    """The covariance has a non-positive pivot, so Eq. 1 is undefined."""


def calibrate(v, gain=None, offset=None) -> np.ndarray:
    """x_b = (v_b - offset_b) * gain_b in FP64 (Sec. 3.2; per-band affine reading)."""
    x = np.asarray(v, dtype=np.float64)
    if offset is not None:
        x = x - np.asarray(offset, dtype=np.float64)
    if gain is not None:
        x = x * np.asarray(gain, dtype=np.float64)
    return x


def gain_correct(v, line_gain) -> np.ndarray:
    """Per-line gain correction (Sec. 3.2): u[t] = v[t] / g_t for lines v [T, ...] and
    gains g [T], in FP64. Pinned by the invariance of scores when each line holds its gain
    times a common scene (tests/test_oracle_pins.py)."""
    v = np.asarray(v, dtype=np.float64)
    g = np.asarray(line_gain, dtype=np.float64).reshape(-1)
    if g.shape[0] != v.shape[0] or not np.all(np.isfinite(g)) or not np.all(g > 0):
        raise ValueError("one finite positive gain per line")
    return v / g.reshape((-1,) + (1,) * (v.ndim - 1))


def sample_mean(X: np.ndarray) -> np.ndarray:
    """Per-band average over all N pixels of X [N, B] (Sec. 3.3)."""
    X = np.asarray(X, dtype=np.float64)
    return X.sum(axis=0) / X.shape[0]


def sample_covariance(X: np.ndarray, mu: np.ndarray) -> np.ndarray:
    """Sigma = sum_p (x_p - mu)(x_p - mu)^T / (N - 1), second pass of two (Sec. 3.3)."""
    X = np.asarray(X, dtype=np.float64)
    D = X - mu
    return (D.T @ D) / (X.shape[0] - 1)


def cholesky_lower(S: np.ndarray) -> np.ndarray:
    """Textbook Cholesky factor L (lower, positive diagonal) with S = L L^T.

    Column j: L_jj = sqrt(S_jj - sum_{k<j} L_jk^2), then
    L_ij = (S_ij - sum_{k<j} L_ik L_jk) / L_jj for i > j.
    Raises NotPositiveDefinite when a pivot is not positive.
    """
    S = np.asarray(S, dtype=np.float64)
    n = S.shape[0]
    L = np.zeros_like(S)
    for j in range(n):
        pivot = S[j, j] - L[j, :j] @ L[j, :j]
        if not (pivot > 0.0) or not math.isfinite(pivot):
            raise NotPositiveDefinite(f"pivot {j} = {pivot!r}")
        L[j, j] = math.sqrt(pivot)
        L[j + 1:, j] = (S[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def forward_substitution(L: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Z with L Z = R for lower-triangular L [B, B] and right-hand sides R [B, n]."""
    L = np.asarray(L, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    Z = np.zeros_like(R)
    for i in range(L.shape[0]):
        Z[i] = (R[i] - L[i, :i] @ Z[:i]) / L[i, i]
    return Z


def rx_scores(S: np.ndarray, mu: np.ndarray, Sigma: np.ndarray) -> np.ndarray:
    """Eq. 1 for every row s of S [n, B]: (s - mu)^T Sigma^{-1} (s - mu) via Cholesky."""
    S = np.asarray(S, dtype=np.float64)
    L = cholesky_lower(Sigma)
    Z = forward_substitution(L, (S - mu).T)
    return (Z * Z).sum(axis=0)


def threshold_mask(delta: np.ndarray, tau: float, mode: str = ABS, delta_max=None) -> np.ndarray:
    """Anomaly mask: delta > tau (ABS) or delta / delta_max > tau (REL). NaN -> False."""
    delta = np.asarray(delta, dtype=np.float64)
    with np.errstate(invalid="ignore"):
        if mode == REL:
            dmax = np.nanmax(delta) if delta_max is None else delta_max
            return (delta / dmax) > tau
        return delta > tau


def global_rx(cube: np.ndarray, gain=None, offset=None):
    """Global RX of one cube [L, W, B] (Sec. 3.3): statistics over all its pixels.

    Returns ``(delta [L, W], delta / max(delta))``.
    """
    L_, W, B = cube.shape
    X = calibrate(cube.reshape(-1, B), gain, offset)
    mu = sample_mean(X)
    Sigma = sample_covariance(X, mu)
    d = rx_scores(X, mu, Sigma).reshape(L_, W)
    return d, d / d.max()


# ---------------------------------------------------------------- streamed forms
LineSource = Union[np.ndarray, Callable[[int, int], np.ndarray]]


def _fetch(lines: LineSource, t0: int, n: int) -> np.ndarray:
    if callable(lines):
        return lines(t0, n)
    return lines[t0:t0 + n]


def statistics_lines(t: int, mode: str, cube_lines: int, n_lines: int, every: int = 1) -> tuple[int, int]:
    """Half-open line range [a, b) whose pixels form the statistics for scoring line t.

    ``every`` (EXCLUSIVE only) is the factorisation cadence: the statistics are taken only
    every ``every`` lines after the reset r, so line t uses the last such snapshot,
    [r, r + every * floor((t - r) / every)); every = 1 is [r, t)."""
    r = (t // cube_lines) * cube_lines if cube_lines > 0 else 0
    if every < 1 or (every > 1 and mode != EXCLUSIVE):
        raise ValueError("a cadence needs EXCLUSIVE statistics and every >= 1")
    if mode == EXCLUSIVE:
        return r, r + every * ((t - r) // every)
    if mode == INCLUSIVE:
        return r, t + 1
    if mode == CUBE:
        if cube_lines <= 0:
            return 0, n_lines
        return r, min(r + cube_lines, n_lines)
    raise ValueError(mode)


def forget_weights(a: int, b: int, lam: float) -> np.ndarray:
    """Per-line weights of window lines [a, b) under exponential forgetting: line tau
    weighs lam^(b - 1 - tau) (the newest line 1). Pinned by exact brute force on
    replicated pixels (tests/test_oracle_pins.py)."""
    return np.asarray([float(lam) ** (b - 1 - tau) for tau in range(a, b)], dtype=np.float64)


def _stats_over_lines(lines: LineSource, a: int, b: int, gain, offset, chunk: int, lam: float = 1.0):
    """Two-pass mean and N-1 covariance over the pixels of lines [a, b), every pixel of
    line tau weighted by forget_weights (all 1 for lam = 1); N is the sum of the weights.

    The sums run over line chunks only to bound host memory; each pass is the
    same sum as the unchunked definition, in a different rounding order.
    """
    w = forget_weights(a, b, lam)
    s1, n = None, 0.0
    for t0 in range(a, b, chunk):
        X = calibrate(_fetch(lines, t0, min(chunk, b - t0)), gain, offset)
        wl = w[t0 - a:t0 - a + X.shape[0]]
        # lam = 1: the plain sum (every weight is 1)
        s = X.reshape(-1, X.shape[-1]).sum(axis=0) if lam == 1.0 else np.einsum("l,lwb->b", wl, X)
        s1 = s if s1 is None else s1 + s
        n += float(wl.sum()) * X.shape[1]
    mu = s1 / n
    m2 = None
    for t0 in range(a, b, chunk):
        X = calibrate(_fetch(lines, t0, min(chunk, b - t0)), gain, offset)
        wl = w[t0 - a:t0 - a + X.shape[0]]
        D = (X - mu).reshape(-1, X.shape[-1])
        c = D.T @ D if lam == 1.0 else (D * np.repeat(wl, X.shape[1])[:, None]).T @ D
        m2 = c if m2 is None else m2 + c
    return mu, m2 / (n - 1), n


def stream_rx_line(lines: LineSource, t: int, mode: str = EXCLUSIVE, cube_lines: int = 0,
                   warmup_pixels: int = 0, gain=None, offset=None, n_lines: int | None = None,
                   chunk: int = 64, every: int = 1, line_gain=None, forget: float = 1.0):
    """Scores of line t under the given statistics window.

    Returns ``(delta [W], status)`` with status OK, NOT_READY (too few pixels;
    delta is NaN) or NOT_PD (covariance not positive definite; delta is NaN).
    ``line_gain`` (one gain per line of ``lines``): every line is gain-corrected
    (``gain_correct``) before the calibration. ``forget`` in (0, 1]: exponential forgetting
    of the streamed window (``forget_weights``).
    """
    if not (0.0 < forget <= 1.0) or (forget < 1.0 and (mode == CUBE or every > 1)):
        raise ValueError("forgetting needs 0 < forget <= 1, streamed statistics and no cadence")
    if line_gain is not None:
        raw, g = lines, np.asarray(line_gain, dtype=np.float64).reshape(-1)

        def lines(t0, n):  # noqa: F811 (the gain-corrected source)
            return gain_correct(_fetch(raw, t0, n), g[t0:t0 + n])

        if n_lines is None:
            n_lines = (t + 1) if callable(raw) else raw.shape[0]
    line = calibrate(_fetch(lines, t, 1), gain, offset)[0]
    W, B = line.shape
    if n_lines is None:
        n_lines = (t + 1) if callable(lines) else lines.shape[0]
    a, b = statistics_lines(t, mode, cube_lines, n_lines, every)
    n_pix = float(forget_weights(a, b, forget).sum()) * W
    if n_pix < max(B + 1, int(warmup_pixels)):
        return np.full(W, np.nan), NOT_READY
    mu, Sigma, _ = _stats_over_lines(lines, a, b, gain, offset, chunk, forget)
    try:
        return rx_scores(line, mu, Sigma), OK
    except NotPositiveDefinite:
        return np.full(W, np.nan), NOT_PD


def stream_rx(lines: np.ndarray, mode: str = EXCLUSIVE, cube_lines: int = 0, warmup_pixels: int = 0,
              gain=None, offset=None, every: int = 1, line_gain=None, forget: float = 1.0):
    """Scores of every line of ``lines`` [T, W, B]: ``(delta [T, W], status [T])``."""
    T, W, B = lines.shape
    delta = np.full((T, W), np.nan)
    status = np.zeros(T, dtype=np.int32)
    for t in range(T):
        delta[t], status[t] = stream_rx_line(lines, t, mode, cube_lines, warmup_pixels,
                                             gain, offset, n_lines=T, every=every, line_gain=line_gain,
                                             forget=forget)
    return delta, status


def encode_tx(scores):
    """Transmit encoding of a block of scores (Sec. 3.4): ``(codes uint16, delta_max)``.

    code = binary16(sqrt(delta / delta_max)) with the division and square root in FP32
    (the paper computes scores in single precision) and round-to-nearest-even to
    binary16; delta_max = the largest finite score (0 if none: every finite score then
    encodes as 0); NaN stays NaN, +Inf encodes as +Inf.
    Pinned by hand-computed binary16 patterns, a nearest-rounding check that decodes the
    codes bit by bit, and monotonicity (tests/test_oracle_pins.py).
    """
    s = np.asarray(scores, dtype=np.float32)
    finite = np.isfinite(s)
    dmax = np.float32(s[finite].max()) if finite.any() else np.float32(0.0)
    with np.errstate(invalid="ignore", divide="ignore"):
        if dmax > 0:
            r = np.sqrt(s / dmax)  # float32 / float32 and float32 sqrt: IEEE, correctly rounded
        else:
            r = np.where(np.isnan(s), np.float32(np.nan), np.where(np.isinf(s), s, np.float32(0.0)))
    return r.astype(np.float32).astype(np.float16).view(np.uint16), float(dmax)


def frontend(raw, first: int, bin_: int, bands: int) -> np.ndarray:
    """Band discard and binning of raw lines [..., B_raw] (Sec. 3.2): the sum of raw bands
    first + bin * b .. first + bin * b + bin - 1 for b = 0 .. bands - 1, as integers.
    Pinned by a hand example and by the band-sum invariant (tests/test_oracle_pins.py)."""
    raw = np.asarray(raw)
    if first < 0 or bin_ < 1 or bands < 1 or first + bin_ * bands > raw.shape[-1]:
        raise ValueError("band range outside the raw line")
    kept = raw[..., first:first + bin_ * bands].astype(np.int64)
    return kept.reshape(raw.shape[:-1] + (bands, bin_)).sum(axis=-1)
