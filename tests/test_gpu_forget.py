"""Exponential forgetting of the streamed statistics on the GPU against the oracle (needs a
GB300).

An extension the paper does not define (reading in the oracle's header): the pixels of a
window line weigh forget^age, the mean is the weighted mean and the covariance the
weighted centred sum over (N - 1), N the sum of the weights. Batches of 7 lines and of 40
lines exercise the carried state and the 32-line scan of the prefix kernels; tolerances
and mask margins are the usual ones.
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


def _lines(T, W, B, seed):
    from gen import PushbroomScene
    sc = PushbroomScene(W, B, seed=seed)
    return sc, sc.lines(0, T)


def _check(s, m, st, ref, rst, prec, B, min_ok=3):
    np.testing.assert_array_equal(st, rst)
    assert (rst == orx.OK).sum() >= min_ok
    emax, _ = rel_err(s, ref)
    assert emax <= TOL[prec], emax
    tau = B + 6 * np.sqrt(2 * B)
    assert mask_mismatch(m, ref, tau, MARGIN[prec]) == 0


@pytest.mark.parametrize("prec,mode,W,B,lam,batch", [
    ("fp32", "exclusive", 130, 270, 0.98, 7), ("bf16", "exclusive", 130, 270, 0.98, 40),
    ("fp32", "inclusive", 65, 64, 0.9, 40), ("bf16", "inclusive", 33, 129, 0.95, 7),
    ("fp16", "exclusive", 64, 96, 0.9, 7), ("bf16", "exclusive", 300, 448, 0.97, 40),
])
def test_forgetting_matches_oracle(hs, prec, mode, W, B, lam, batch):
    T = 40
    sc, lines = _lines(T, W, B, seed=W + B)
    det = hs.Detector(width=W, bands=B, precision=prec, stats_mode=mode, forget=lam, max_batch_lines=batch)
    first = det.push(lines)
    rc, s, m, st = det.scores(first, T)
    det.close()
    ref, rst = orx.stream_rx(lines, getattr(oracle, mode.upper()), gain=sc.gain, offset=sc.offset,
                             forget=float(np.float32(lam)))
    _check(s, m, st, ref, rst, prec, B)


def test_forgetting_float_input_and_resets(hs):
    rng = np.random.default_rng(3)
    T, W, B = 30, 40, 20
    lines = (rng.normal(size=(T, W, B)) @ np.diag(np.linspace(0.5, 2.0, B)) + 3.0).astype(np.float32)
    det = hs.Detector(width=W, bands=B, in_dtype="f32", precision="fp32", forget=0.8, cube_lines=12,
                      max_batch_lines=5)
    first = det.push(lines)
    rc, s, m, st = det.scores(first, T)
    det.close()
    ref, rst = orx.stream_rx(lines, oracle.EXCLUSIVE, cube_lines=12, forget=float(np.float32(0.8)))
    _check(s, m, st, ref, rst, "fp32", B)


def test_forgetting_with_gains_and_batch_invariance(hs):
    W, B, T = 96, 130, 24
    sc, lines = _lines(T, W, B, seed=77)
    g = np.random.default_rng(77).uniform(0.8, 1.25, size=T).astype(np.float32)
    out = []
    for batch in (4, 24):
        det = hs.Detector(width=W, bands=B, precision="bf16", forget=0.95, max_batch_lines=batch)
        first = det.push(lines, gains=g)
        rc, s, m, st = det.scores(first, T)
        det.close()
        out.append(s)
    ref, rst = orx.stream_rx(lines, oracle.EXCLUSIVE, line_gain=g.astype(np.float64),
                             forget=float(np.float32(0.95)))
    _check(out[0], m, st, ref, rst, "bf16", B)
    np.testing.assert_allclose(out[1], out[0], rtol=1e-5, atol=1e-5)


def test_forget_one_is_the_plain_stream(hs):
    sc, lines = _lines(10, 64, 70, seed=5)
    res = []
    for kw in ({}, dict(forget=1.0)):
        det = hs.Detector(width=64, bands=70, precision="bf16", **kw)
        first = det.push(lines)
        res.append(det.scores(first, 10)[1])
        det.close()
    np.testing.assert_array_equal(res[0], res[1])


def test_forgetting_window_that_never_fills_and_no_export(hs):
    rng = np.random.default_rng(9)
    lines = rng.integers(100, 200, size=(30, 2, 3)).astype(np.uint16)
    det = hs.Detector(width=2, bands=3, forget=0.5)          # N < W / (1 - 0.5) = 4 = B + 1
    first = det.push(lines)
    rc, s, m, st = det.scores(first, 30)
    assert rc == hs.HSAD_E_NOT_READY and (st == 1).all() and np.isnan(s).all() and not m.any()
    assert hs.hsad_get_stats(det.ctx, 3)[0] == hs.HSAD_E_INVALID
    det.close()
