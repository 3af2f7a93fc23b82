"""FP64 oracle of subsampled kernel RX (test infrastructure; never called by the library).

Sec. 2.2 ("Detection Algorithm", Table tab:results) compares global RX with subsampled
kernel RX, citing the kernel RX of Kwon and Nasrabadi (2005) and the subsampled, faster
form of Hidalgo et al. (2021); the paper prints neither formula nor parameters, so this
module writes out kernel RX from its published definition, with these readings:

* Kernel RX: RX (Eq. 1) of the pixels mapped into the feature space of a kernel k. With
  the background samples s_1..s_m mapped and centred in that space, the feature-space
  covariance is C = Phi~ Phi~^T / (m - 1) (the unbiased denominator of the RX reading,
  Sec. 3.3), and by the kernel trick the score of a pixel r is
      delta(r) = (m - 1) * k~_r^T (K~)^+2 k~_r,
  K~ = H K H the centred Gram matrix of the background (H = I - 1 1^T / m) and
  k~_r = H (k_r - K 1 / m) the centred kernel vector of r, (k_r)_i = k(s_i, r).
* Regularisation: K~ is singular (rank <= m - 1), and kernel RX inverts it only through a
  regularised form. Reading: (K~)^+2 -> (K~ + lam I)^-2 with lam = eps * trace(K~) / m,
      delta(r) = (m - 1) * || (K~ + lam I)^{-1} k~_r ||^2.
* Kernel: the Gaussian radial basis function k(x, y) = exp(-||x - y||^2 / c) of kernel RX;
  c = 0 selects the mean squared distance between distinct background samples. The linear
  kernel k(x, y) = x^T y is also provided: with it kernel RX is RX of the background
  samples (the pin below).
* Subsampling: the background is m pixels of the cube chosen at random without
  replacement (the indices are an input, drawn by the caller); every pixel of the cube is
  scored against it (global form, Sec. 3.3).
* Calibration: the kernel sees the calibrated values x_b = (v_b - offset_b) * gain_b of
  Sec. 3.2. Unlike RX, the Gaussian kernel is not invariant under per-band gains; it is
  under translations (offsets) and orthogonal maps of the bands.

Steps per pixel, in the order above: kernel vector, centring, the solve with the Cholesky
factor of K~ + lam I (forward then backward substitution), squared norm times (m - 1).

Pins (tests/test_oracle_krx.py): the linear kernel reduces to RX of the background
samples (rx.rx_scores) as eps -> 0; a two-sample, one-band closed form; the in-sample
identity sum_i delta(s_i) = (m - 1) sum_j l_j^2 / (l_j + lam)^2 over the eigenvalues l_j
of K~ (an eigendecomposition, independent of the Cholesky path); invariance of the
Gaussian-kernel scores under translations and orthogonal maps of the bands; and planted
mistakes (uncentred test vector, K~^-1 instead of K~^-2, m instead of m - 1, a wrong
kernel width) that these pins reject.
"""
from __future__ import annotations

import numpy as np

from .rx import calibrate, cholesky_lower, forward_substitution

RBF, LINEAR = "rbf", "linear"


def squared_distances(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """D_ij = sum_b (x_ib - y_jb)^2 for rows of X [n, B] and Y [m, B], summed term by term."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    D = np.empty((X.shape[0], Y.shape[0]))
    for j in range(Y.shape[0]):
        d = X - Y[j]
        D[:, j] = (d * d).sum(axis=1)
    return D


def mean_pairwise_distance(S: np.ndarray) -> float:
    """c = mean of ||s_i - s_j||^2 over the pairs i < j of the background samples."""
    m = S.shape[0]
    D = squared_distances(S, S)
    return float(D[np.triu_indices(m, 1)].mean())


def kernel_matrix(X: np.ndarray, Y: np.ndarray, kernel: str, c: float) -> np.ndarray:
    """k(x_i, y_j) for the Gaussian RBF exp(-||x - y||^2 / c) or the linear kernel x^T y."""
    if kernel == RBF:
        return np.exp(-squared_distances(X, Y) / c)
    if kernel == LINEAR:
        return np.asarray(X, dtype=np.float64) @ np.asarray(Y, dtype=np.float64).T
    raise ValueError(f"unknown kernel {kernel!r}")


def centering_matrix(m: int) -> np.ndarray:
    """H = I - 1 1^T / m."""
    return np.eye(m) - np.full((m, m), 1.0 / m)


def centered_gram(K: np.ndarray) -> np.ndarray:
    """K~ = H K H: the Gram matrix of the feature vectors minus their mean."""
    H = centering_matrix(K.shape[0])
    return H @ K @ H


def centered_test_vectors(Kr: np.ndarray, K: np.ndarray) -> np.ndarray:
    """Rows k~_r = H (k_r - K 1 / m) for the rows k_r of Kr [n, m]: the inner products of
    the centred feature vector of r with the centred background feature vectors."""
    m = K.shape[0]
    H = centering_matrix(m)
    kbar = K.sum(axis=1) / m
    return (Kr - kbar[None, :]) @ H.T


def backward_substitution(U: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Y with U Y = R for upper-triangular U [m, m] and right-hand sides R [m, n]."""
    U = np.asarray(U, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    Y = np.zeros_like(R)
    for i in range(U.shape[0] - 1, -1, -1):
        Y[i] = (R[i] - U[i, i + 1:] @ Y[i + 1:]) / U[i, i]
    return Y


def krx_background(S: np.ndarray, kernel: str = RBF, c: float = 0.0, eps: float = 1e-3):
    """Everything kernel RX needs from the background samples S [m, B]: the kernel width c,
    the Gram matrix K, the ridge lam and the Cholesky factor of K~ + lam I."""
    S = np.asarray(S, dtype=np.float64)
    m = S.shape[0]
    if m < 2:
        raise ValueError("kernel RX needs at least two background samples")
    if kernel == RBF and c <= 0.0:
        c = mean_pairwise_distance(S)
    K = kernel_matrix(S, S, kernel, c)
    Kc = centered_gram(K)
    lam = eps * np.trace(Kc) / m
    L = cholesky_lower(Kc + lam * np.eye(m))
    return dict(S=S, m=m, c=c, K=K, Kc=Kc, lam=lam, L=L, kernel=kernel)


def krx_scores(R: np.ndarray, bg: dict, chunk: int = 4096) -> np.ndarray:
    """delta(r) = (m - 1) || (K~ + lam I)^{-1} k~_r ||^2 for every row r of R [n, B]."""
    R = np.asarray(R, dtype=np.float64)
    out = np.empty(R.shape[0])
    L, m = bg["L"], bg["m"]
    for a in range(0, R.shape[0], chunk):
        Kr = kernel_matrix(R[a:a + chunk], bg["S"], bg["kernel"], bg["c"])
        kt = centered_test_vectors(Kr, bg["K"])                   # [n, m]
        z = forward_substitution(L, kt.T)                          # L z = k~
        y = backward_substitution(L.T, z)                          # L^T y = z
        out[a:a + chunk] = (m - 1) * (y * y).sum(axis=0)
    return out


def subsampled_krx(cube: np.ndarray, idx, kernel: str = RBF, c: float = 0.0, eps: float = 1e-3,
                   gain=None, offset=None):
    """Global subsampled kernel RX of a cube [..., B]: background = the calibrated pixels at
    the flat indices ``idx``; returns (scores shaped like the cube's pixels, the background
    dict)."""
    X = calibrate(np.asarray(cube).reshape(-1, np.asarray(cube).shape[-1]), gain, offset)
    idx = np.asarray(idx, dtype=np.int64)
    if idx.ndim != 1 or len(np.unique(idx)) != idx.size or idx.min() < 0 or idx.max() >= X.shape[0]:
        raise ValueError("background indices must be distinct pixel indices")
    bg = krx_background(X[idx], kernel, c, eps)
    return krx_scores(X, bg).reshape(np.asarray(cube).shape[:-1]), bg
