"""CPU checks of the split-precision schemes the tensor-core kernels rely on (no GPU).

The kernels compute exact or extended-precision products from BF16 tensor-core products:

* the FP32 whitening operand is split into three BF16 terms hi + mid + lo, each the BF16
  rounding of the FP32 remainder of the ones before (claimed exact: their sum is the FP32
  value);
* the factor's float-float rows are split into six signed base-256 digits with a per-row
  power of two (Ozaki et al.'s error-free splitting): every digit an integer of magnitude
  <= 256 (exact in BF16), the value recovered to 2^e 256^-6 / 2, the 64-term level sums of
  digit products below 2^24 (exact in FP32), and a product of two split rows within about
  2^-45 of the row scales.

These emulate the arithmetic with numpy (FP32 rounding where the kernels round in FP32, BF16
rounding by round-to-nearest-even to 8 significant bits) and check those claims on seeded
random data, including rows with a wide spread of magnitudes.
"""
import numpy as np
import pytest


def bf16(x):
    """Round float32 values to the nearest BF16 (ties to even), returned as float32."""
    x = np.asarray(x, dtype=np.float32)
    b = x.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def split3(v):
    """hi, mid, lo as in the kernels' three-plane operands and operand splits."""
    v = np.asarray(v, dtype=np.float32)
    hi = bf16(v)
    r = (v - hi).astype(np.float32)
    mid = bf16(r)
    lo = bf16((r - mid).astype(np.float32))
    return hi, mid, lo


def test_three_term_bf16_split_is_exact():
    rng = np.random.default_rng(1)
    v = np.concatenate([rng.standard_normal(200000).astype(np.float32),
                        (rng.standard_normal(20000) * 10.0 ** rng.uniform(-20, 20, 20000)).astype(np.float32)])
    hi, mid, lo = split3(v)
    # each term is a BF16 value
    for t in (hi, mid, lo):
        np.testing.assert_array_equal(t, bf16(t))
    # (hi + mid) + lo in FP32 is the value itself
    s = ((hi + mid).astype(np.float32) + lo).astype(np.float32)
    np.testing.assert_array_equal(s, v)
    # and exactly in FP64
    np.testing.assert_array_equal(hi.astype(np.float64) + mid + lo, v.astype(np.float64))


def test_six_term_products_drop_only_fp32_rounding_order_terms():
    """The FP32 whitening keeps the products a_t h_u with t + u <= 2 of three-term splits:
    the dropped terms are below about 3 * 2^-24 of |a| |h|."""
    rng = np.random.default_rng(2)
    a = rng.standard_normal(100000).astype(np.float32)
    h = (rng.standard_normal(100000) * 10.0 ** rng.uniform(-3, 3, 100000)).astype(np.float32)
    A, H = split3(a), split3(h)
    kept = sum(A[t].astype(np.float64) * H[u] for t in range(3) for u in range(3) if t + u <= 2)
    exact = a.astype(np.float64) * h.astype(np.float64)
    err = np.abs(kept - exact) / (np.abs(a.astype(np.float64)) * np.abs(h.astype(np.float64)))
    assert err.max() <= 3 * 2.0 ** -24


def split_digits_rows(hi, lo, ndig=6):
    """Per-row exponent and six base-256 digits of float-float rows (hi + lo), as the factor's
    kernels do: e from the row's largest |hi| (|v| <= mx < 2^e), then per digit x *= 256,
    d = rint(x), x -= d with the float-float remainder renormalised in FP32."""
    hi = np.asarray(hi, dtype=np.float32)
    lo = np.asarray(lo, dtype=np.float32)
    mx = np.abs(hi).max(axis=1)
    e = np.where(mx > 0, np.frexp(mx)[1], 0).astype(np.int64)
    sc = np.ldexp(np.float32(1.0), -e).astype(np.float32)[:, None]
    xh = (hi * sc).astype(np.float32)
    xl = (lo * sc).astype(np.float32)
    digits = []
    for _ in range(ndig):
        xh = (xh * np.float32(256)).astype(np.float32)
        xl = (xl * np.float32(256)).astype(np.float32)
        d = np.rint(xh).astype(np.float32)
        s = (xh - d).astype(np.float32)  # exact
        # two-sum of s and xl, as ff_norm
        h2 = (s + xl).astype(np.float32)
        z = (h2 - s).astype(np.float32)
        l2 = ((s - (h2 - z)).astype(np.float32) + (xl - z).astype(np.float32)).astype(np.float32)
        xh, xl = h2, l2
        digits.append(d)
    return e, digits


def ff_rows(rng, n, m, spread):
    """Float-float rows: FP64 values with magnitudes spread over `spread` decades."""
    v = rng.standard_normal((n, m)) * 10.0 ** rng.uniform(-spread, 0, (n, m))
    v *= 10.0 ** rng.uniform(-5, 5, (n, 1))
    hi = v.astype(np.float32)
    lo = (v - hi.astype(np.float64)).astype(np.float32)
    return hi, lo, hi.astype(np.float64) + lo.astype(np.float64)


@pytest.mark.parametrize("spread", [0.0, 3.0, 8.0])
def test_six_digit_split_recovers_rows_and_sums_exactly(spread):
    rng = np.random.default_rng(3 + int(spread))
    n, m = 96, 64
    hi, lo, v = ff_rows(rng, n, m, spread)
    e, dg = split_digits_rows(hi, lo)
    # digits are integers of magnitude <= 256, hence exact in BF16
    for d in dg:
        assert np.all(d == np.rint(d)) and np.abs(d).max() <= 256
        np.testing.assert_array_equal(bf16(d), d)
    # the value is recovered to 2^e 256^-6 / 2 (plus the float-float pair's own 2^-48)
    rec = sum(d.astype(np.float64) * 256.0 ** -(t + 1) for t, d in enumerate(dg)) * np.ldexp(1.0, e)[:, None]
    bound = np.ldexp(1.0, e)[:, None] * (256.0 ** -6 / 2) + np.abs(v) * 2.0 ** -47
    assert np.all(np.abs(rec - v) <= bound)
    # the level sums of a product of two split row sets over 64 terms stay below 2^24
    e2, dg2 = split_digits_rows(*ff_rows(rng, n, m, spread)[:2])
    for lvl in range(6):
        S = sum(dg[t].astype(np.float64) @ dg2[lvl - t].astype(np.float64).T for t in range(lvl + 1))
        assert np.abs(S).max() < 2.0 ** 24
        # and FP32 accumulation of the terms in any order is exact: every partial sum is an
        # integer below 2^24
        np.testing.assert_array_equal(S.astype(np.float32).astype(np.float64), S)


def test_six_digit_products_are_within_two_to_minus_45_of_the_row_scales():
    """sum_l 256^-l S_l * 2^(e_i + e_j - 16) against the exact product of the float-float
    rows: within a few 2^-45 * 2^e_i * 2^e_j per 64-term product."""
    rng = np.random.default_rng(7)
    n, m = 128, 64
    hA, lA, A = ff_rows(rng, n, m, 4.0)
    hB, lB, Bm = ff_rows(rng, 64, m, 4.0)
    eA, dA = split_digits_rows(hA, lA)
    eB, dB = split_digits_rows(hB, lB)
    S = [sum(dA[t].astype(np.float64) @ dB[l - t].astype(np.float64).T for t in range(l + 1)) for l in range(6)]
    approx = sum(S[l] * 256.0 ** -l for l in range(6)) * np.ldexp(1.0, eA[:, None] + eB[None, :] - 16)
    exact = A @ Bm.T
    scale = np.ldexp(1.0, eA[:, None] + eB[None, :])
    rel = np.abs(approx - exact) / scale
    assert rel.max() <= 8 * 2.0 ** -45, rel.max()  # dropping level 5 gives ~150 x 2^-45
