"""Front end (Sec. 3.2: band discard and binning) on the GPU against the oracle (needs a GB300).

Binning is integer work, so the binned lines and the covariance sums built from them must
be bit-exact; the binned 12-bit DN reach 14 bits, which the exact tensor-core SYRK handles
with 256-pixel slices (lines wider than that exercise the sliced accumulation). Scores
follow the usual tolerances against the oracle applied to the oracle's own binning.
"""
import numpy as np
import pytest

import oracle
from oracle import rx as orx
from tests._parity import MARGIN, TOL, mask_mismatch, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_13509_gb300 as hs
    return hs


def _raw(T, W, raw_bands, seed):
    from gen import PushbroomScene
    return PushbroomScene(W, raw_bands, seed=seed).lines(0, T)   # 12-bit DN


@pytest.mark.parametrize("first,bin_,bands", [(0, 1, 300), (10, 4, 70), (3, 3, 99), (1, 2, 149)])
def test_frontend_kernel_bit_exact(hs, first, bin_, bands):
    import torch
    raw = _raw(3, 77, 300, seed=first + 10 * bin_)
    n = raw.shape[0] * raw.shape[1]
    d_raw = torch.from_numpy(raw.view(np.int16)).cuda()
    d_out = torch.empty((n, bands), dtype=torch.int16, device="cuda")
    assert hs.hsad_frontend(d_raw, n, 300, first, bin_, bands, d_out) == hs.HSAD_OK
    ref = oracle.frontend(raw, first, bin_, bands).reshape(n, bands)
    np.testing.assert_array_equal(d_out.cpu().numpy().view(np.uint16).astype(np.int64), ref)
    assert hs.hsad_frontend(d_raw, n, 300, 250, 4, 70, d_out) == hs.HSAD_E_INVALID   # past the raw bands


def _exact_sums(binned):
    x0 = binned[0].astype(np.int64)
    c = np.rint(x0.sum(axis=0) / x0.shape[0]).astype(np.int64)
    X = binned.reshape(-1, binned.shape[-1]).astype(np.int64) - c
    return c, X.sum(axis=0), X.T @ X


@pytest.mark.parametrize("W,mem", [(96, "host"), (640, "device"), (640, "pinned")])
def test_frontend_stream_sums_bit_exact(hs, W, mem):
    import torch
    raw = _raw(7, W, 300, seed=W + 1)
    det = hs.Detector(width=W, bands=70, stats_mode="exclusive", raw_bands=300, band_first=10, band_bin=4,
                      max_batch_lines=3)
    if mem == "device":
        det.push(torch.from_numpy(raw.view(np.int16)).cuda())
    elif mem == "pinned":
        det.push(torch.from_numpy(raw.view(np.int16)).pin_memory())
    else:
        det.push(raw)
    rc, n, c, s1, s2 = hs.hsad_get_stats(det.ctx, 70)
    det.close()
    binned = oracle.frontend(raw, 10, 4, 70)
    ce, s1e, s2e = _exact_sums(binned)
    assert rc == hs.HSAD_OK and n == 7 * W
    np.testing.assert_array_equal(c, ce.astype(np.float64))
    np.testing.assert_array_equal(s1, s1e.astype(np.float64))
    lo = np.tril_indices(70)
    np.testing.assert_array_equal(s2[lo], s2e[lo].astype(np.float64))


@pytest.mark.parametrize("prec,mode", [("fp32", "exclusive"), ("bf16", "exclusive"), ("fp32", "cube")])
def test_frontend_scores_match_oracle(hs, prec, mode):
    raw = _raw(24, 300, 300, seed=7)
    binned = oracle.frontend(raw, 10, 4, 70)
    kw = dict(cube_lines=12) if mode == "cube" else {}
    det = hs.Detector(width=300, bands=70, stats_mode=mode, precision=prec, raw_bands=300, band_first=10,
                      band_bin=4, max_batch_lines=5, **kw)
    first = det.push(raw)
    rc, s, m, st = det.scores(first, 24)
    det.close()
    ref, rst = orx.stream_rx(binned, getattr(oracle, mode.upper()), **kw)
    np.testing.assert_array_equal(st, rst)
    emax, _ = rel_err(s, ref)
    assert emax <= TOL[prec], emax
    tau = 70 + 6 * np.sqrt(140)
    assert mask_mismatch(m, ref, tau, MARGIN[prec]) == 0
