"""Failure detection without a GPU fault.

A device wait that can never complete gives up after its limit and reports a timeout
that the host reads; the device stays usable afterwards. Host-side failures (bad
arguments, results that were never pushed, polling before completion) return status
codes and leave the context working.
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


def test_bounded_device_wait_times_out_and_device_stays_usable(hs):
    rc, flag = hs.hsad_selftest_bounded_wait(0, 2_000_000)     # about 1 ms of SM clocks
    assert rc == hs.HSAD_E_TIMEOUT and flag == 1
    # the device and the library still work afterwards
    from gen import PushbroomScene
    sc = PushbroomScene(64, 16, seed=1)
    lines = sc.lines(0, 10)
    det = hs.Detector(width=64, bands=16, precision="bf16")
    first = det.push(lines)
    rc, s, m, st = det.scores(first, 10)
    det.close()
    assert np.isfinite(s[1:]).all()


def test_host_side_failures_leave_context_usable(hs):
    from gen import PushbroomScene
    sc = PushbroomScene(48, 12, seed=2)
    lines = sc.lines(0, 8)
    det = hs.Detector(width=48, bands=12)
    s = np.empty((4, 48), np.float32)
    assert hs.hsad_scores(det.ctx, 0, 4, s, None, hs.HSAD_HOST, 0) == hs.HSAD_E_INVALID   # nothing pushed
    assert hs.hsad_push_lines(det.ctx, lines, -1, hs.HSAD_HOST)[0] == hs.HSAD_E_INVALID
    assert hs.hsad_push_lines(det.ctx, lines, 8, 7)[0] == hs.HSAD_E_INVALID
    first = det.push(lines)
    rc, s8, m8, st = det.scores(first, 8)
    assert rc in (hs.HSAD_OK, hs.HSAD_E_NOT_READY) and np.isfinite(s8[1:]).all()
    det.close()
