"""Per-line gain correction (Sec. 3.2) on the GPU against the oracle (needs a GB300).

The imager changes its gain for every line and the data is corrected for it before the
calibration: line t is scored as DN / g_t. The lines below are the synthetic scene
recorded at a per-line gain (DN = round(g_t x scene), clipped to 12 bits) and pushed with
those gains through hsad_push_lines_gain; the oracle divides every line by its gain
(``line_gain`` of ``oracle.stream_rx``). Tolerances and mask margins are the usual ones.
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


def _gained_lines(T, W, B, seed, lo=0.7, hi=1.3):
    from gen import PushbroomScene
    sc = PushbroomScene(W, B, seed=seed)
    scene = sc.lines(0, T).astype(np.float64)
    g = np.random.default_rng(seed).uniform(lo, hi, size=T).astype(np.float32)
    dn = np.clip(np.rint(scene * g.astype(np.float64)[:, None, None]), 0, 4095).astype(np.uint16)
    return sc, dn, g


def _check(s, m, st, ref, rst, prec, B):
    np.testing.assert_array_equal(st, rst)
    assert (rst == orx.OK).sum() >= 3
    emax, _ = rel_err(s, ref)
    assert emax <= TOL[prec], emax
    tau = B + 6 * np.sqrt(2 * B)
    assert mask_mismatch(m, ref, tau, MARGIN[prec]) == 0


@pytest.mark.parametrize("prec,mode,W,B", [("fp32", "exclusive", 130, 270), ("bf16", "exclusive", 130, 270),
                                           ("fp32", "inclusive", 65, 64), ("bf16", "inclusive", 33, 129),
                                           ("bf16", "exclusive", 300, 448), ("fp32", "exclusive", 7, 3)])
def test_gain_stream_matches_oracle(hs, prec, mode, W, B):
    T = max(8, (B + 1) // W + 6)
    sc, dn, g = _gained_lines(T, W, B, seed=W * 7 + B)
    det = hs.Detector(width=W, bands=B, precision=prec, stats_mode=mode, max_batch_lines=5)
    first = det.push(dn, gains=g)
    rc, s, m, st = det.scores(first, T)
    det.close()
    ref, rst = orx.stream_rx(dn, getattr(oracle, mode.upper()), gain=sc.gain, offset=sc.offset,
                             line_gain=g.astype(np.float64))
    _check(s, m, st, ref, rst, prec, B)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_gain_batches_pinned_device_and_mixed_pushes(hs, prec):
    """Batch boundaries, device and pinned pushes, and pushes without gains (gain 1) mixed
    with pushes with gains all give the oracle's scores."""
    import torch
    W, B, T = 96, 130, 16
    sc, dn, g = _gained_lines(T, W, B, seed=5)
    g_mixed = g.copy()
    g_mixed[:4] = 1.0
    dn[:4] = np.clip(np.rint(sc.lines(0, 4).astype(np.float64)), 0, 4095).astype(np.uint16)
    ref, rst = orx.stream_rx(dn, oracle.EXCLUSIVE, line_gain=g_mixed.astype(np.float64))
    out = []
    for how in ("pieces", "device", "pinned"):
        det = hs.Detector(width=W, bands=B, precision=prec, max_batch_lines=4)
        first = det.push(dn[:4])                                    # no gains: gain 1
        if how == "pieces":
            det.push(dn[4:7], gains=g_mixed[4:7])
            det.push(dn[7:], gains=g_mixed[7:])
        elif how == "device":
            det.push(torch.from_numpy(dn[4:].view(np.int16)).cuda(), gains=g_mixed[4:])
        else:
            det.push(torch.from_numpy(dn[4:].view(np.int16)).pin_memory(), gains=g_mixed[4:])
        rc, s, m, st = det.scores(first, T)
        det.close()
        _check(s, m, st, ref, rst, prec, B)
        out.append(s)
    np.testing.assert_allclose(out[1], out[0], rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(out[2], out[0], rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_gain_recovers_the_scene(hs, prec):
    """Each line holds its gain (1 or 2) times the scene exactly: with the gains its scores
    are the scene's own, and without them they are not."""
    from gen import PushbroomScene
    W, B, T = 64, 96, 12
    scene = PushbroomScene(W, B, seed=31).lines(0, T) // 2                     # 11-bit scene
    g = np.random.default_rng(31).choice([1.0, 2.0], size=T).astype(np.float32)
    dn = (scene.astype(np.int64) * g.astype(np.int64)[:, None, None]).astype(np.uint16)
    ref, rst = orx.stream_rx(scene, oracle.EXCLUSIVE)
    det = hs.Detector(width=W, bands=B, precision=prec)
    first = det.push(dn, gains=g)
    rc, s, m, st = det.scores(first, T)
    det.close()
    _check(s, m, st, ref, rst, prec, B)
    raw, _ = orx.stream_rx(dn, oracle.EXCLUSIVE)
    ok = rst == orx.OK
    assert np.nanmax(np.abs(raw[ok] - ref[ok]) / np.maximum(ref[ok], 1.0)) > 10 * TOL[prec]


def test_gain_with_front_end(hs):
    """Gains of binned lines: the raw lines' gain carries over to their band sums."""
    from gen import PushbroomScene
    W, T = 120, 10
    raw = PushbroomScene(W, 300, seed=8).lines(0, T)
    g = np.random.default_rng(8).uniform(0.8, 1.25, size=T).astype(np.float32)
    det = hs.Detector(width=W, bands=70, precision="bf16", raw_bands=300, band_first=10, band_bin=4,
                      max_batch_lines=4)
    first = det.push(raw, gains=g)
    rc, s, m, st = det.scores(first, T)
    det.close()
    binned = oracle.frontend(raw, 10, 4, 70)
    ref, rst = orx.stream_rx(binned, oracle.EXCLUSIVE, line_gain=g.astype(np.float64))
    _check(s, m, st, ref, rst, "bf16", 70)


def test_gain_push_rejections(hs):
    W, B = 16, 8
    lines = np.full((3, W, B), 100, dtype=np.uint16)
    ok_g = np.ones(3, dtype=np.float32)
    for kw in (dict(stats_mode="cube", cube_lines=4), dict(in_dtype="f32"), dict(precision="fp16")):
        det = hs.Detector(width=W, bands=B, **kw)
        x = lines.astype(np.float32) if kw.get("in_dtype") == "f32" else lines
        rc, _ = hs.hsad_push_lines_gain(det.ctx, x, ok_g, 3, hs.HSAD_HOST)
        assert rc == hs.HSAD_E_INVALID, kw
        det.close()
    det = hs.Detector(width=W, bands=B)
    for bad in (0.0, -1.0, np.nan, np.inf, 1e6):
        g = ok_g.copy()
        g[1] = bad
        rc, _ = hs.hsad_push_lines_gain(det.ctx, lines, g, 3, hs.HSAD_HOST)
        assert rc == hs.HSAD_E_INVALID, bad
    rc, _ = hs.hsad_push_lines_gain(det.ctx, lines, None, 3, hs.HSAD_HOST)
    assert rc == hs.HSAD_E_INVALID
    rc, first = hs.hsad_push_lines_gain(det.ctx, lines, ok_g, 3, hs.HSAD_HOST)
    assert rc == hs.HSAD_OK and first == 0                     # nothing was enqueued before
    det.close()
