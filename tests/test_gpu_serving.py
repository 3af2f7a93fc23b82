"""Serving engine: each stream's results are the same alone and in the mix; admission by budget.

Streams of different widths and band counts run concurrently through one engine; lines
are submitted interleaved and in uneven groups, so the worker batches them differently
from a stand-alone context. The per-line arithmetic does not depend on batching (the
covariance sums are exact integers), so the scores must agree to the last bit.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_13509_gb300 as hs
    return hs


SHAPES = [(96, 40, "bf16"), (130, 64, "fp32"), (64, 129, "fp16")]


def _alone(hs, lines, sc, prec):
    det = hs.Detector(width=lines.shape[1], bands=lines.shape[2], precision=prec, gain=sc.gain, offset=sc.offset)
    first = det.push(lines)
    rc, s, m, st = det.scores(first, lines.shape[0])
    det.close()
    return s, m


def test_results_identical_alone_and_in_mix(hs):
    from gen import PushbroomScene
    T = 40
    data = []
    for k, (W, B, prec) in enumerate(SHAPES):
        sc = PushbroomScene(W, B, seed=500 + k)
        data.append((sc, sc.lines(0, T), prec))
    rc, eng = hs.hsad_engine_create(0, 0)
    assert rc == hs.HSAD_OK
    sids = []
    for sc, lines, prec in data:
        cfg = hs.make_config(lines.shape[1], lines.shape[2], precision=prec, gain=sc.gain, offset=sc.offset,
                             max_batch_lines=8)
        rc, sid = hs.hsad_engine_open(eng, cfg)
        assert rc == hs.HSAD_OK
        sids.append(sid)
    # interleaved submissions of uneven sizes
    rng = np.random.default_rng(0)
    pos = [0] * len(data)
    while any(p < T for p in pos):
        k = int(rng.integers(0, len(data)))
        if pos[k] >= T:
            continue
        n = int(min(T - pos[k], rng.integers(1, 6)))
        rc, first = hs.hsad_engine_submit(eng, sids[k], np.ascontiguousarray(data[k][1][pos[k]:pos[k] + n]), n)
        assert rc == hs.HSAD_OK and first == pos[k]
        pos[k] += n
    for k, (sc, lines, prec) in enumerate(data):
        s = np.empty((T, lines.shape[1]), np.float32)
        m = np.empty((T, lines.shape[1]), np.uint8)
        rc = hs.hsad_engine_results(eng, sids[k], 0, T, s, m, 20000)
        assert rc in (hs.HSAD_OK, hs.HSAD_E_NOT_READY), hs.hsad_status_string(rc)
        s0, m0 = _alone(hs, lines, sc, prec)
        np.testing.assert_array_equal(np.isnan(s), np.isnan(s0))
        np.testing.assert_array_equal(np.nan_to_num(s), np.nan_to_num(s0))
        np.testing.assert_array_equal(m, m0)
    rc, n_lines, n_push, max_batch = hs.hsad_engine_counters(eng)
    assert rc == hs.HSAD_OK and n_lines == 3 * T and n_push < 3 * T
    assert hs.hsad_engine_destroy(eng) == hs.HSAD_OK


def test_admission_by_device_budget(hs):
    import gc
    gc.collect()                                           # contexts of earlier tests released
    base = hs.hsad_device_budget_used(0)
    cfg = hs.make_config(256, 128, max_batch_lines=16)
    det = hs.Detector(width=256, bands=128, max_batch_lines=16)
    need = det.device_bytes
    det.close()
    rc, eng = hs.hsad_engine_create(0, int(base + need * 1.5))   # room for one stream, not two
    assert rc == hs.HSAD_OK
    rc, a = hs.hsad_engine_open(eng, cfg)
    assert rc == hs.HSAD_OK
    rc, b = hs.hsad_engine_open(eng, cfg)
    assert rc == hs.HSAD_E_BUSY
    assert hs.hsad_engine_close(eng, a) == hs.HSAD_OK
    rc, b = hs.hsad_engine_open(eng, cfg)
    assert rc == hs.HSAD_OK
    big = hs.make_config(4096, 512, max_batch_lines=4096)
    rc, c = hs.hsad_engine_open(eng, big)
    assert rc == hs.HSAD_E_NOMEM                           # can never fit this budget
    hs.hsad_engine_destroy(eng)
    hs.hsad_set_device_budget(0, 0)
    assert hs.hsad_device_budget_used(0) == base


def test_stream_closed_mid_flight_leaves_the_others_intact(hs):
    """Closing a stream while its lines are queued and on the GPU waits (bounded) for its
    work, frees its budget and returns OK; the other stream's results are unaffected, and
    destroying a plain context with work in flight also returns OK."""
    from gen import PushbroomScene
    gc_base = hs.hsad_device_budget_used(0)
    scs = [PushbroomScene(128, 96, seed=600), PushbroomScene(96, 40, seed=601)]
    lines = [sc.lines(0, 60) for sc in scs]
    rc, eng = hs.hsad_engine_create(0, 0)
    assert rc == hs.HSAD_OK
    sids = []
    for sc, ln in zip(scs, lines):
        cfg = hs.make_config(ln.shape[1], ln.shape[2], precision="bf16", gain=sc.gain, offset=sc.offset,
                             max_batch_lines=8)
        rc, sid = hs.hsad_engine_open(eng, cfg)
        assert rc == hs.HSAD_OK
        sids.append(sid)
    for t in range(0, 60, 3):  # both streams busy
        for k in range(2):
            assert hs.hsad_engine_submit(eng, sids[k], np.ascontiguousarray(lines[k][t:t + 3]), 3)[0] == hs.HSAD_OK
    assert hs.hsad_engine_close(eng, sids[0]) == hs.HSAD_OK          # mid-flight
    assert hs.hsad_engine_submit(eng, sids[0], np.ascontiguousarray(lines[0][:1]), 1)[0] == hs.HSAD_E_INVALID
    s = np.empty((60, 96), np.float32)
    m = np.empty((60, 96), np.uint8)
    rc = hs.hsad_engine_results(eng, sids[1], 0, 60, s, m, 20000)
    assert rc in (hs.HSAD_OK, hs.HSAD_E_NOT_READY), hs.hsad_status_string(rc)
    s0, m0 = _alone(hs, lines[1], scs[1], "bf16")
    np.testing.assert_array_equal(np.nan_to_num(s), np.nan_to_num(s0))
    np.testing.assert_array_equal(m, m0)
    assert hs.hsad_engine_destroy(eng) == hs.HSAD_OK
    # a plain context destroyed with pushed, unread work in flight
    det = hs.Detector(width=128, bands=96, precision="bf16", gain=scs[0].gain, offset=scs[0].offset)
    det.push(lines[0])
    assert hs.hsad_destroy(det.ctx) == hs.HSAD_OK
    det.ctx = None
    assert hs.hsad_device_budget_used(0) == gc_base


def test_front_end_and_cadence_streams_in_the_mix(hs):
    """A front-end stream (raw 120-band lines binned to 28) and a cadence stream (k = 3) run
    beside a plain one; each gives the results of the same configuration alone."""
    from gen import PushbroomScene
    T = 30
    raw = PushbroomScene(72, 120, seed=61).lines(0, T)
    sc2 = PushbroomScene(80, 32, seed=62)
    plain = sc2.lines(0, T)
    kws = [dict(width=72, bands=28, raw_bands=120, band_first=4, band_bin=4),
           dict(width=80, bands=32, factor_every=3, gain=sc2.gain, offset=sc2.offset),
           dict(width=80, bands=32, precision="bf16", gain=sc2.gain, offset=sc2.offset)]
    inputs = [raw, plain, plain]
    rc, eng = hs.hsad_engine_create(0, 0)
    assert rc == hs.HSAD_OK
    sids = []
    for kw in kws:
        rc, sid = hs.hsad_engine_open(eng, hs.make_config(max_batch_lines=8, **kw))
        assert rc == hs.HSAD_OK, hs.hsad_status_string(rc)
        sids.append(sid)
    rng = np.random.default_rng(3)
    pos = [0] * 3
    while any(p < T for p in pos):
        k = int(rng.integers(0, 3))
        if pos[k] >= T:
            continue
        n = int(min(T - pos[k], rng.integers(1, 5)))
        rc, first = hs.hsad_engine_submit(eng, sids[k], np.ascontiguousarray(inputs[k][pos[k]:pos[k] + n]), n)
        assert rc == hs.HSAD_OK and first == pos[k]
        pos[k] += n
    for k, kw in enumerate(kws):
        W = kw["width"]
        s = np.empty((T, W), np.float32)
        m = np.empty((T, W), np.uint8)
        rc = hs.hsad_engine_results(eng, sids[k], 0, T, s, m, 20000)
        assert rc in (hs.HSAD_OK, hs.HSAD_E_NOT_READY), hs.hsad_status_string(rc)
        det = hs.Detector(**kw)
        first = det.push(inputs[k])
        _, s0, m0, _ = det.scores(first, T)
        det.close()
        np.testing.assert_array_equal(np.nan_to_num(s, nan=-1.0), np.nan_to_num(s0, nan=-1.0))
        np.testing.assert_array_equal(m, m0)
    assert hs.hsad_engine_destroy(eng) == hs.HSAD_OK
