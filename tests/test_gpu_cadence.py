"""Factorisation cadence (an extension: EXCLUSIVE statistics snapshot every k lines) on the
GPU against the oracle (needs a GB300).

Line t is scored against the statistics of lines [r, r + k floor((t - r) / k)). The library
factors only the snapshot slots of each batch and carries the last one across batches, so
batch sizes that do not divide k, statistics resets, CUDA-graph replay and a statistics
import at a snapshot must all give the oracle's scores, and the same scores whatever the
batching (bitwise).
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


@pytest.mark.parametrize("k,prec,batch,cube_lines", [(2, "fp32", 3, 0), (3, "bf16", 4, 0), (5, "fp32", 7, 11),
                                                     (4, "bf16", 1, 0)])
def test_cadence_matches_oracle(hs, k, prec, batch, cube_lines):
    sc, lines = _lines(33, 80, 24, seed=100 + k)
    det = hs.Detector(width=80, bands=24, stats_mode="exclusive", precision=prec, gain=sc.gain, offset=sc.offset,
                      max_batch_lines=batch, cube_lines=cube_lines, factor_every=k)
    det.push(lines)
    rc, s, m, st = det.scores(0, 33)
    det.close()
    ref, rst = orx.stream_rx(lines, oracle.EXCLUSIVE, cube_lines=cube_lines, gain=sc.gain, offset=sc.offset,
                             every=k)
    np.testing.assert_array_equal(st, rst)
    emax, _ = rel_err(s, ref)
    assert emax <= TOL[prec], emax
    assert mask_mismatch(m, ref, 24 + 6 * np.sqrt(48), MARGIN[prec]) == 0


def test_cadence_is_batch_and_graph_invariant(hs):
    sc, lines = _lines(40, 64, 20, seed=77)
    out = []
    for pushes, flags in (([40], 0), ([1, 2, 3, 1, 5, 2, 7, 1, 4, 14], hs.HSAD_CUDA_GRAPHS),
                          ([3] * 13 + [1], hs.HSAD_CUDA_GRAPHS)):
        det = hs.Detector(width=64, bands=20, stats_mode="exclusive", gain=sc.gain, offset=sc.offset,
                          max_batch_lines=8, factor_every=3, flags=flags)
        t = 0
        for n in pushes:
            det.push(lines[t:t + n])
            t += n
        rc, s, m, st = det.scores(0, 40)
        det.close()
        out.append((s, m, st))
    for s, m, st in out[1:]:
        np.testing.assert_array_equal(np.nan_to_num(s, nan=-1.0), np.nan_to_num(out[0][0], nan=-1.0))
        np.testing.assert_array_equal(m, out[0][1])
        np.testing.assert_array_equal(st, out[0][2])


def test_cadence_of_one_is_every_line(hs):
    sc, lines = _lines(20, 48, 16, seed=5)
    res = []
    for every in (0, 1):
        det = hs.Detector(width=48, bands=16, stats_mode="exclusive", factor_every=every, max_batch_lines=6)
        det.push(lines)
        res.append(det.scores(0, 20)[1])
        det.close()
    np.testing.assert_array_equal(np.nan_to_num(res[0], nan=-1.0), np.nan_to_num(res[1], nan=-1.0))


def test_cadence_statistics_import_at_a_snapshot(hs):
    sc, lines = _lines(18, 40, 12, seed=9)
    full = hs.Detector(width=40, bands=12, stats_mode="exclusive", factor_every=3, max_batch_lines=4)
    full.push(lines)
    ref = full.scores(0, 18)[1]
    full.close()
    a = hs.Detector(width=40, bands=12, stats_mode="exclusive", factor_every=3, max_batch_lines=4)
    a.push(lines[:9])                                   # 9 lines: a snapshot (multiple of 3)
    rc, n, c, s1, s2 = hs.hsad_get_stats(a.ctx, 12)
    a.close()
    b = hs.Detector(width=40, bands=12, stats_mode="exclusive", factor_every=3, max_batch_lines=4)
    assert hs.hsad_set_stats(b.ctx, n, c, s1, s2) == hs.HSAD_OK
    first = b.push(lines[9:])
    rc, s, m, st = b.scores(first, 9)
    b.close()
    np.testing.assert_array_equal(np.nan_to_num(s, nan=-1.0), np.nan_to_num(ref[9:], nan=-1.0))
    d = hs.Detector(width=40, bands=12, stats_mode="exclusive", factor_every=3)
    assert hs.hsad_set_stats(d.ctx, 40 * 8, c, s1, s2) == hs.HSAD_E_INVALID   # 8 lines: not a snapshot
    d.close()
