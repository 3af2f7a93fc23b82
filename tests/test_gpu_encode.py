"""Transmit encoding (Sec. 3.4) on the GPU against the oracle (needs a GB300).

The encoding is integer-valued (binary16 codes), so given the same FP32 scores both sides
must agree bit for bit; against the oracle's own FP64 scores the codes may differ by one
unit in the last place where a score's rounding error crosses a binary16 rounding boundary.
"""
import numpy as np
import pytest

import oracle
from oracle import rx as orx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_13509_gb300 as hs
    return hs


def _scores(seed, n):
    rng = np.random.default_rng(seed)
    s = rng.gamma(0.6, 40.0, n).astype(np.float32)
    s[::97] = 0.0
    s[5::131] = np.nan
    if n > 13:
        s[7] = np.float32(1e-30)
        s[11] = np.float32(3e-8)        # ratios below the binary16 normal range
        s[13] = np.nanmax(s)            # a repeated maximum
    return s


@pytest.mark.parametrize("n", [1, 257, 100_003])
def test_encode_scores_bit_exact(hs, n):
    import torch
    s = _scores(n, n)
    ds = torch.from_numpy(s).cuda()
    dc = torch.empty(n, dtype=torch.int16, device="cuda")
    rc, mx = hs.hsad_encode_scores(ds, n, dc)
    assert rc == hs.HSAD_OK
    codes = dc.cpu().numpy().view(np.uint16)
    ref, rmax = oracle.encode_tx(s)
    assert np.float32(mx) == np.float32(rmax)
    np.testing.assert_array_equal(codes, ref)


def test_encode_scores_special_blocks(hs):
    import torch
    for s in (np.array([np.nan, np.nan], np.float32), np.zeros(5, np.float32),
              np.array([0.0, np.inf, 2.0, np.nan], np.float32)):
        ds = torch.from_numpy(s).cuda()
        dc = torch.empty(len(s), dtype=torch.int16, device="cuda")
        rc, mx = hs.hsad_encode_scores(ds, len(s), dc)
        ref, rmax = oracle.encode_tx(s)
        assert rc == hs.HSAD_OK and np.float32(mx) == np.float32(rmax)
        np.testing.assert_array_equal(dc.cpu().numpy().view(np.uint16), ref)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_scores_tx_of_a_stream(hs, prec):
    from gen import PushbroomScene
    sc = PushbroomScene(96, 24, seed=41)
    lines = sc.lines(0, 30)
    # a 16-line result ring: the requested block wraps around it
    det = hs.Detector(width=96, bands=24, stats_mode="exclusive", precision=prec, gain=sc.gain,
                      offset=sc.offset, result_lines=16, max_batch_lines=8)
    det.push(lines[:14])
    det.push(lines[14:])                # the ring now holds lines 14..29 in slots 14, 15, 0..13
    rc, s, m, st = det.scores(14, 14)
    rc2, codes, mx = det.scores_tx(14, 14)
    import torch
    dcodes = torch.empty((14, 96), dtype=torch.int16, device="cuda")
    rc3, mx3 = hs.hsad_scores_tx(det.ctx, 14, 14, dcodes, hs.HSAD_DEVICE, -1)
    det.close()
    assert rc == rc2 == rc3 == hs.HSAD_OK
    # the library's own FP32 scores encode bit for bit like the oracle's encoding of them
    ref, rmax = oracle.encode_tx(s)
    assert np.float32(mx) == np.float32(rmax) == np.float32(mx3)
    np.testing.assert_array_equal(codes, ref)
    np.testing.assert_array_equal(dcodes.cpu().numpy().view(np.uint16), ref)
    # against the oracle's scores: at most one unit in the last place apart
    dref, _ = orx.stream_rx(lines, oracle.EXCLUSIVE, gain=sc.gain, offset=sc.offset)
    cref, _ = oracle.encode_tx(dref[14:28])
    diff = np.abs(codes.astype(np.int64) - cref.astype(np.int64))
    assert diff.max() <= 1
    if prec == "fp32":
        assert (diff == 0).mean() >= 0.99


def test_scores_tx_warmup_lines_are_nan_and_cube_max_is_one(hs):
    from gen import PushbroomScene
    sc = PushbroomScene(40, 20, seed=43)
    lines = sc.lines(0, 12)
    det = hs.Detector(width=40, bands=20, stats_mode="exclusive", gain=sc.gain, offset=sc.offset)
    det.push(lines)
    rc, codes, mx = det.scores_tx(0, 12)
    rcs, s, m, st = det.scores(0, 12)
    det.close()
    assert rc == rcs == hs.HSAD_E_NOT_READY            # line 0 has no statistics yet
    assert (codes[st != 0] == 0x7E00).all()
    ok = np.isfinite(s)
    assert codes[ok].max() == 0x3C00 and np.float32(mx) == np.float32(s[ok].max())

    # CUBE mode, one whole cube requested: the paper's per-cube normalisation
    det = hs.Detector(width=40, bands=20, stats_mode="cube", cube_lines=12, gain=sc.gain, offset=sc.offset)
    det.push(lines)
    rc, codes, mx = det.scores_tx(0, 12)
    det.close()
    ref, _ = orx.stream_rx(lines, oracle.CUBE, cube_lines=12, gain=sc.gain, offset=sc.offset)
    cref, rmax = oracle.encode_tx(ref)
    assert rc == hs.HSAD_OK and abs(mx - rmax) <= 1e-4 * rmax
    assert np.abs(codes.astype(np.int64) - cref.astype(np.int64)).max() <= 1
