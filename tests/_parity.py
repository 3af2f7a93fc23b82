"""Shared comparison helpers for the GPU parity tests (no RX arithmetic here)."""
import numpy as np

# Tolerances on the score: e = |delta - delta_ref| / max(delta_ref, 1).
TOL = {"fp32": 1e-4, "bf16": 1e-2, "fp16": 1e-2}
# Mask margin: pixels with |delta_ref - tau| <= m * tau may disagree.
MARGIN = {"fp32": 2e-4, "bf16": 2e-2, "fp16": 2e-2}


def rel_err(d, ref):
    d = np.asarray(d, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    ok = np.isfinite(ref)
    assert np.array_equal(np.isfinite(d), ok), "NaN pattern differs from the oracle"
    if not ok.any():
        return 0.0, 0.0
    e = np.abs(d[ok] - ref[ok]) / np.maximum(ref[ok], 1.0)
    return float(e.max()), float(np.percentile(e, 99.9))


def mask_mismatch(mask, ref_value, tau, margin):
    """Pixels whose mask differs from (ref_value > tau) outside the margin band."""
    ref_value = np.asarray(ref_value, dtype=np.float64)
    with np.errstate(invalid="ignore"):
        ref = ref_value > tau
        band = np.abs(ref_value - tau) <= margin * tau
    ref = np.where(np.isfinite(ref_value), ref, False)
    bad = (np.asarray(mask).astype(bool) != ref) & ~band
    return int(bad.sum())
