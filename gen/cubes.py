"""Seeded synthetic push-broom hyperspectral data.

The paper's flight data (VNIR push-broom imager, 900 samples x 300 bands per
line, 12-bit DN, 1000-line cubes; Sec. 3.2 "Data Acquisition") is not
available, so every input is drawn here from a fixed recipe:

* ``GaussianMixtureCube`` -- a small float32 reflectance cube: a 4-component
  Gaussian mixture laid out as a Voronoi map, with 2x2 implanted anomalies at
  10 % mixing. Used for global (per-cube) RX, Sec. 3.3.
* ``PushbroomScene`` -- an unbounded stream of uint16 12-bit DN lines:
  radiance = illumination x reflectance of 6 materials whose abundances drift
  along track, Poisson shot noise plus Gaussian read noise, a per-band dark
  offset, and 0.1 % anomalous pixels in clusters of 1-9 pixels.

Every random draw comes from a Philox counter-based generator keyed by
``(seed, stream, block)``, so any line range can be regenerated on its own and
the result does not depend on how many threads generate it.

Nothing in this module computes a statistic of the data.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

SEED_BASE = 20260213
BLOCK_LINES = 64          # lines drawn per independent generator block
FULL_SCALE = 4095         # 12-bit sensor


def rng_for(seed: int, *keys: int) -> np.random.Generator:
    """Philox4x32-10 generator keyed by (seed, *keys)."""
    ss = np.random.SeedSequence([int(seed)] + [int(k) for k in keys])
    return np.random.Generator(np.random.Philox(ss))


def smooth_spectrum(rng: np.random.Generator, bands: int, lo: float = 0.05,
                    hi: float = 0.6, bumps: int = 3) -> np.ndarray:
    """Sum of Gaussian bumps over the band index, mapped affinely onto [lo, hi]."""
    if bands == 1:
        rng.uniform(size=3 * bumps)  # keep the draw count independent of B
        return np.array([(lo + hi) / 2.0])
    b = np.arange(bands, dtype=np.float64)
    c = rng.uniform(0.0, bands, bumps)
    w = np.maximum(rng.uniform(bands / 12.0, bands / 3.0, bumps), 0.75)
    a = rng.uniform(0.2, 1.0, bumps)
    s = (a[:, None] * np.exp(-0.5 * ((b[None, :] - c[:, None]) / w[:, None]) ** 2)).sum(0)
    span = s.max() - s.min()
    if span <= 0:
        return np.full(bands, (lo + hi) / 2.0)
    return lo + (hi - lo) * (s - s.min()) / span


def haar_orthogonal(rng: np.random.Generator, n: int) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of a Gaussian matrix, signs fixed."""
    g = rng.standard_normal((n, n))
    q, r = np.linalg.qr(g)
    return q * np.where(np.diag(r) < 0, -1.0, 1.0)[None, :]


class GaussianMixtureCube:
    """Float32 reflectance cube with implanted anomalies (global RX workload).

    Background: ``n_components`` Gaussian components with weights ``weights``
    assigned to the cells of a seeded Voronoi map; component k has a smooth
    mean spectrum in [0.05, 0.6] and covariance U_k diag(lam) U_k^T with U_k
    Haar and lam_i = sigma^2 * 10^(-decades * i / (B-1)). sigma = 0.003 was
    calibrated once so that the implanted anomalies rank above the background
    under exact global RX (median anomaly score above the background's 99th
    percentile, AUC >= 0.99), then frozen.
    Anomalies: ``n_anomalies`` non-overlapping 2x2 blocks whose pixels are
    (1-mix) * background + mix * a_j for a distinct smooth spectrum a_j.
    """

    def __init__(self, lines=64, width=128, bands=64, seed=SEED_BASE + 1,
                 n_components=4, weights=(0.4, 0.3, 0.2, 0.1), n_cells=12,
                 sigma=0.003, decades=3.0, n_anomalies=20, anomaly_mix=0.1):
        self.lines, self.width, self.bands = int(lines), int(width), int(bands)
        self.seed = int(seed)
        self.n_components = int(n_components)
        self.weights = np.asarray(weights, dtype=np.float64)
        self.n_cells = int(n_cells)
        self.sigma, self.decades = float(sigma), float(decades)
        self.n_anomalies, self.anomaly_mix = int(n_anomalies), float(anomaly_mix)

    def generate(self):
        """Return ``(cube float32 [L,W,B], anomaly bool [L,W], label int [L,W])``."""
        L, W, B, K = self.lines, self.width, self.bands, self.n_components
        rng = rng_for(self.seed, 0)
        means = np.stack([smooth_spectrum(rng, B) for _ in range(K)])
        i = np.arange(B, dtype=np.float64)
        expo = self.decades * i / (B - 1) if B > 1 else np.zeros(1)
        lam = self.sigma ** 2 * 10.0 ** (-expo)
        U = np.stack([haar_orthogonal(rng, B) for _ in range(K)])

        sites = np.stack([rng.uniform(0, L, self.n_cells), rng.uniform(0, W, self.n_cells)], 1)
        cell_comp = rng.choice(K, size=self.n_cells, p=self.weights / self.weights.sum())
        yy, xx = np.meshgrid(np.arange(L) + 0.5, np.arange(W) + 0.5, indexing="ij")
        d2 = (yy[..., None] - sites[:, 0]) ** 2 + (xx[..., None] - sites[:, 1]) ** 2
        label = cell_comp[np.argmin(d2, axis=-1)]

        z = rng.standard_normal((L, W, B)) * np.sqrt(lam)
        cube = np.empty((L, W, B), dtype=np.float64)
        for k in range(K):
            sel = label == k
            cube[sel] = means[k] + z[sel] @ U[k].T

        anomaly = np.zeros((L, W), dtype=bool)
        if L >= 2 and W >= 2 and self.n_anomalies > 0:
            spectra = np.stack([smooth_spectrum(rng, B) for _ in range(self.n_anomalies)])
            placed, tries = 0, 0
            while placed < self.n_anomalies and tries < 100000:
                tries += 1
                r0 = int(rng.integers(0, L - 1))
                c0 = int(rng.integers(0, W - 1))
                if anomaly[r0:r0 + 2, c0:c0 + 2].any():
                    continue
                anomaly[r0:r0 + 2, c0:c0 + 2] = True
                blk = cube[r0:r0 + 2, c0:c0 + 2]
                cube[r0:r0 + 2, c0:c0 + 2] = (1 - self.anomaly_mix) * blk + self.anomaly_mix * spectra[placed]
                placed += 1
        return cube.astype(np.float32), anomaly, label


def config1_cube():
    """64 lines x 128 pixels x 64 bands float32 mixture cube (seed 20260213+1)."""
    return GaussianMixtureCube(64, 128, 64, seed=SEED_BASE + 1).generate()


class PushbroomScene:
    """Unbounded stream of uint16 12-bit DN push-broom lines, BIP layout [line][pixel][band].

    Per pixel (t = line, x = sample):
      abundances  w = softmax(a_k + b_k sin(2 pi t / T_k + phi_k)
                              + c_k sin(2 pi f_k x / W + psi_k) + 1.2 n),  n ~ N(0, 1)
      reflectance r = w @ R  (R: 6 smooth material spectra in [0.05, 0.6]);
                  0.1 % of pixels, in clusters of 1-9, are mixed with one of
                  4 anomaly spectra at a fraction in [0.3, 0.7]
      signal      s_b = A * I_b * r_b * (1 + 0.05 sin(2 pi t / 2500 + rho))   [DN]
      DN          clamp(rint(off_b + q_b * Poisson(s_b / q_b) + N(0, read_noise)), 0, 4095)
    with I the illumination spectrum (smooth, with absorption dips near 760 and
    940 nm), q_b in [0.3, 0.6] DN per photo-electron, off_b in [50, 150] DN and
    A chosen so the brightest band sits at 60-80 % of full scale.
    ``gain`` and ``offset`` map DN back to approximate reflectance:
    (DN - offset_b) * gain_b.
    """

    def __init__(self, width: int, bands: int, seed: int, n_materials: int = 6,
                 anomaly_fraction: float = 1e-3, read_noise: float = 2.0):
        self.width, self.bands, self.seed = int(width), int(bands), int(seed)
        self.anomaly_fraction, self.read_noise = float(anomaly_fraction), float(read_noise)
        B = self.bands
        rng = rng_for(self.seed, 0)
        wl = np.linspace(400.0, 1000.0, B) if B > 1 else np.array([700.0])
        self.wavelength = wl
        illum = np.exp(-0.5 * ((wl - 600.0) / 220.0) ** 2)
        illum *= 1.0 - 0.5 * np.exp(-0.5 * ((wl - 760.0) / 6.0) ** 2)
        illum *= 1.0 - 0.6 * np.exp(-0.5 * ((wl - 940.0) / 25.0) ** 2)
        self.illum = illum + 0.05
        self.materials = np.stack([smooth_spectrum(rng, B) for _ in range(n_materials)])
        self.a = rng.normal(0.0, 1.0, n_materials)
        self.b = rng.uniform(0.5, 1.5, n_materials)
        self.period = rng.uniform(1500.0, 6000.0, n_materials)
        self.phase = rng.uniform(0.0, 2 * np.pi, n_materials)
        self.c = rng.uniform(0.3, 1.0, n_materials)
        self.xfreq = rng.uniform(0.5, 3.0, n_materials)
        self.xphase = rng.uniform(0.0, 2 * np.pi, n_materials)
        self.rho = rng.uniform(0.0, 2 * np.pi)
        self.offset = rng.uniform(50.0, 150.0, B)
        self.q = rng.uniform(0.3, 0.6, B)
        self.anomaly_spectra = np.stack([smooth_spectrum(rng, B, 0.02, 0.9, bumps=5) for _ in range(4)])
        peak = float((self.illum * self.materials.max(0)).max())
        self.amplitude = rng.uniform(0.6, 0.8) * (FULL_SCALE - self.offset.max()) / peak / 1.05
        self.gain = 1.0 / (self.amplitude * self.illum)

    # -- one independent block of BLOCK_LINES lines ---------------------------------
    def _block(self, k: int):
        W, B, nl = self.width, self.bands, BLOCK_LINES
        rng = rng_for(self.seed, 1, k)
        t = (k * nl + np.arange(nl, dtype=np.float64))[:, None, None]
        x = np.arange(W, dtype=np.float64)[None, :, None]
        logits = (self.a + self.b * np.sin(2 * np.pi * t / self.period + self.phase)
                  + self.c * np.sin(2 * np.pi * self.xfreq * x / W + self.xphase)
                  + 1.2 * rng.standard_normal((nl, W, self.a.size)))
        logits -= logits.max(-1, keepdims=True)
        w = np.exp(logits)
        w /= w.sum(-1, keepdims=True)
        refl = w @ self.materials                                   # [nl, W, B]

        mask = np.zeros((nl, W), dtype=bool)
        n_clusters = int(rng.poisson(self.anomaly_fraction * nl * W / 5.0))
        for _ in range(n_clusters):
            tc, xc = int(rng.integers(0, nl)), int(rng.integers(0, W))
            size = int(rng.integers(1, 10))
            spec = self.anomaly_spectra[int(rng.integers(0, 4))]
            frac = rng.uniform(0.3, 0.7)
            for o in rng.permutation(9)[:size]:
                dt, dx = divmod(int(o), 3)
                tt, xx = tc + dt - 1, xc + dx - 1
                if 0 <= tt < nl and 0 <= xx < W and not mask[tt, xx]:
                    refl[tt, xx] = (1 - frac) * refl[tt, xx] + frac * spec
                    mask[tt, xx] = True

        drift = 1.0 + 0.05 * np.sin(2 * np.pi * t / 2500.0 + self.rho)
        signal = self.amplitude * self.illum * refl * drift          # DN above dark offset
        electrons = rng.poisson(signal / self.q)
        dn = self.offset + self.q * electrons + rng.normal(0.0, self.read_noise, signal.shape)
        return np.clip(np.rint(dn), 0, FULL_SCALE).astype(np.uint16), mask

    def _blocks(self, t0: int, n: int, threads):
        k0, k1 = t0 // BLOCK_LINES, (t0 + n + BLOCK_LINES - 1) // BLOCK_LINES
        ks = list(range(k0, k1))
        threads = threads or min(len(ks), max(1, (os.cpu_count() or 1)), 16)
        if threads <= 1 or len(ks) <= 1:
            return ks, [self._block(k) for k in ks]
        with ThreadPoolExecutor(threads) as ex:
            return ks, list(ex.map(self._block, ks))

    def lines(self, t0: int, n: int, out: np.ndarray | None = None, threads: int | None = None):
        """DN of lines [t0, t0+n) as uint16 [n, W, B] (written into ``out`` if given)."""
        if out is None:
            out = np.empty((n, self.width, self.bands), dtype=np.uint16)
        if n == 0:
            return out
        k0 = t0 // BLOCK_LINES
        # generate in bounded groups so peak host memory stays modest
        group = 32
        for g0 in range(0, (t0 + n + BLOCK_LINES - 1) // BLOCK_LINES - k0, group):
            ga = (k0 + g0) * BLOCK_LINES
            gb = min((k0 + g0 + group) * BLOCK_LINES, t0 + n)
            lo = max(ga, t0)
            ks, blocks = self._blocks(lo, gb - lo, threads)
            for k, (dn, _) in zip(ks, blocks):
                a, b = max(k * BLOCK_LINES, lo), min((k + 1) * BLOCK_LINES, gb)
                out[a - t0:b - t0] = dn[a - k * BLOCK_LINES:b - k * BLOCK_LINES]
        return out

    def anomaly_mask(self, t0: int, n: int):
        """Ground-truth anomaly mask of lines [t0, t0+n) as bool [n, W]."""
        out = np.zeros((n, self.width), dtype=bool)
        ks, blocks = self._blocks(t0, n, None)
        for k, (_, m) in zip(ks, blocks):
            a, b = max(k * BLOCK_LINES, t0), min((k + 1) * BLOCK_LINES, t0 + n)
            if a < b:
                out[a - t0:b - t0] = m[a - k * BLOCK_LINES:b - k * BLOCK_LINES]
        return out


class IllConditionedScene:
    """Lines whose band covariance has a prescribed, very large condition number.

    Every pixel is ``2048 + U diag(a) z`` (DN units) with U a Haar orthogonal B x B matrix,
    z ~ N(0, I_B) drawn per pixel and a_j = 500 sqrt(B) 10^(-decades j / (B - 1)): the
    bands are strongly correlated (about 500 DN of spread per band along the leading
    direction) and the population covariance U diag(a^2) U^T has condition number
    10^(2 decades). ``dtype="f32"``: the values divided by 4096, as float32 (nothing else
    bounds the conditioning); ``dtype="u16"``: rounded and clamped 12-bit DN, where the
    rounding noise (variance 1/12 per band) caps the sample covariance's condition number
    near 10^6. No anomalies are implanted. Stands in for a scene dominated by one material
    under a low-noise sensor, the hardest case for the factorisation.
    """

    def __init__(self, width: int, bands: int, seed: int, decades: float = 5.0, dtype: str = "f32"):
        self.width, self.bands, self.seed = int(width), int(bands), int(seed)
        self.decades, self.dtype = float(decades), dtype
        B = self.bands
        self.U = haar_orthogonal(rng_for(self.seed, 0), B)
        self.a = 500.0 * np.sqrt(B) * 10.0 ** (-self.decades * np.arange(B) / max(B - 1, 1))
        self.gain = None
        self.offset = None

    def lines(self, t0: int, n: int) -> np.ndarray:
        """Lines [t0, t0 + n) as [n, W, B] float32 or uint16 (one generator block per line)."""
        W, B = self.width, self.bands
        out = np.empty((n, W, B), dtype=np.float64)
        for i in range(n):
            z = rng_for(self.seed, 1, t0 + i).standard_normal((W, B))
            out[i] = 2048.0 + (z * self.a) @ self.U.T
        if self.dtype == "u16":
            return np.clip(np.rint(out), 0, FULL_SCALE).astype(np.uint16)
        return (out / 4096.0).astype(np.float32)


def subsample_indices(n_pixels: int, m: int, seed: int) -> np.ndarray:
    """m distinct pixel indices in [0, n_pixels), uniform without replacement, sorted: the
    random background subsample of subsampled kernel RX (drawn here, passed to both sides)."""
    if not 0 < m <= n_pixels:
        raise ValueError("need 0 < m <= n_pixels")
    return np.sort(rng_for(seed, 2).choice(n_pixels, size=m, replace=False)).astype(np.int64)


# Named workloads (seed SEED_BASE + k for workload k).
SCENES = {
    "stream_640x270": dict(width=640, bands=270, lines=4000, seed=SEED_BASE + 2),
    "precision_1024x448": dict(width=1024, bands=448, lines=8000, seed=SEED_BASE + 3),
}


def config_scene(name: str):
    """Return ``(scene, n_lines)`` for a named stream workload."""
    p = SCENES[name]
    return PushbroomScene(p["width"], p["bands"], p["seed"]), p["lines"]


def serving_streams(n_streams: int = 16, seed: int = SEED_BASE + 4):
    """16-stream serving mix: widths {320,640,1024}, bands {128,270,448}, Poisson rates U[100,300] lines/s."""
    rng = rng_for(seed, 0)
    out = []
    for i in range(n_streams):
        W = (320, 640, 1024)[i % 3]
        B = (128, 270, 448)[(i // 3) % 3]
        rate = float(rng.uniform(100.0, 300.0))
        out.append(dict(width=W, bands=B, rate=rate, seed=seed * 100 + i))
    return out


def stress_cubes(n_cubes: int = 32, seed: int = SEED_BASE + 5):
    """Uneven stored cubes: W in [2048,4096], B in [224,448], L in [2000,10000]."""
    rng = rng_for(seed, 0)
    return [dict(width=int(rng.integers(2048, 4097)), bands=int(rng.integers(224, 449)),
                 lines=int(rng.integers(2000, 10001)), seed=seed * 100 + i) for i in range(n_cubes)]
