"""The allocation-free global-RX call against the context-based API (needs a GB300).

hsad_global_rx_noalloc serves callers that cannot allocate device memory: it keeps
its intermediates in one static device array instead. Its scores and mask must
agree with a CUBE-mode context scoring the same cube, on two calls in a row (the
second call reuses the array with the first call's contents still in it), also when the
earlier call left a larger layout (more lines, more bands, another padded width) or
stopped at a warm-up status. This file is collected last on purpose.
"""
import numpy as np
import pytest

from tests._parity import MARGIN, TOL, mask_mismatch, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_13509_gb300 as hs
    return hs


def _context_scores(hs, cube, dtype, prec, gain, mode, tau, flags):
    import torch
    det = hs.Detector(width=cube.shape[1], bands=cube.shape[2], in_dtype=dtype, precision=prec,
                      stats_mode="cube", cube_lines=cube.shape[0], gain=gain, threshold_mode=mode,
                      threshold=tau, flags=flags)
    first = det.push(torch.from_numpy(cube).cuda())
    rc, s, m, st = det.scores(first, cube.shape[0])
    det.close()
    return rc, s, m


def _noalloc(hs, cube, dtype, prec, gain, mode, tau, flags):
    import torch
    x = torch.from_numpy(cube).cuda()
    s = torch.full((cube.shape[0], cube.shape[1]), -1.0, dtype=torch.float32, device="cuda")
    m = torch.full((cube.shape[0], cube.shape[1]), 7, dtype=torch.uint8, device="cuda")
    rc = hs.hsad_global_rx_noalloc(x, cube.shape[0], cube.shape[1], cube.shape[2],
                                   hs.HSAD_F32 if dtype == "f32" else hs.HSAD_U16,
                                   {"fp32": hs.HSAD_FP32, "bf16": hs.HSAD_BF16, "fp16": hs.HSAD_FP16}[prec],
                                   gain, hs.HSAD_REL if mode == "rel" else hs.HSAD_ABS, tau, flags, s, m, None, 0)
    torch.cuda.synchronize()
    return rc, s.cpu().numpy(), m.cpu().numpy()


def _cases():
    from gen import PushbroomScene, config1_cube
    cube, _, _ = config1_cube()
    sc = PushbroomScene(96, 40, seed=31)
    dn = sc.lines(0, 50)
    return [
        ("f32-rel", cube, "f32", "fp32", None, "rel", 0.110, 0),
        ("u16-abs", dn.view(np.int16), "u16", "fp32", sc.gain, "abs", 0.0, 0),
        ("u16-bf16-norm", dn.view(np.int16), "u16", "bf16", sc.gain, "rel", 0.110, 2),
    ]


@pytest.mark.parametrize("case", range(3))
def test_noalloc_matches_context_api_twice(hs, case):
    name, cube, dtype, prec, gain, mode, tau, flags = _cases()[case]
    rc0, s0, m0 = _context_scores(hs, cube, dtype, prec, gain, mode, tau, flags)
    assert rc0 == hs.HSAD_OK, name
    for call in range(2):
        rc, s, m = _noalloc(hs, cube, dtype, prec, gain, mode, tau, flags)
        assert rc == hs.HSAD_OK, (name, call, hs.hsad_status_string(rc))
        emax, _ = rel_err(s, s0)
        assert emax <= TOL[prec], (name, call, emax)
        if mode == "abs":
            t = 40 + 6 * np.sqrt(80) if tau == 0.0 else tau
            assert mask_mismatch(m, s0, t, MARGIN[prec]) == 0
        elif flags:
            assert mask_mismatch(m, s0, tau, 2 * MARGIN[prec]) == 0
        else:
            assert mask_mismatch(m, s0 / np.nanmax(s0), tau, 2 * MARGIN[prec]) == 0


def test_noalloc_rejects_oversize_and_bad_arguments(hs):
    import torch
    x = torch.zeros((4, 8, 512), dtype=torch.int16, device="cuda")
    s = torch.zeros((4, 8), dtype=torch.float32, device="cuda")
    m = torch.zeros((4, 8), dtype=torch.uint8, device="cuda")
    # 4000 lines of 512 bands need about 33 MiB of scratch: rejected before any launch
    assert hs.hsad_global_rx_noalloc(x, 4000, 8, 512, hs.HSAD_U16, hs.HSAD_FP32, None, hs.HSAD_ABS, 0.0, 0,
                                     s, m, None, 0) == hs.HSAD_E_INVALID
    assert hs.hsad_global_rx_noalloc(x, 4, 8, 513, hs.HSAD_U16, hs.HSAD_FP32, None, hs.HSAD_ABS, 0.0, 0,
                                     s, m, None, 0) == hs.HSAD_E_INVALID
    assert hs.hsad_global_rx_noalloc(None, 4, 8, 512, hs.HSAD_U16, hs.HSAD_FP32, None, hs.HSAD_ABS, 0.0, 0,
                                     s, m, None, 0) == hs.HSAD_E_INVALID


def test_noalloc_startup_warmup_call(hs):
    """n_lines = 0 only sets the device up (module load, array address) and succeeds with
    every pointer NULL; a bad device is still rejected."""
    assert hs.hsad_global_rx_noalloc(None, 0, 0, 0, 0, 0, None, 0, 0.0, 0, None, None, None, 0) == hs.HSAD_OK
    assert hs.hsad_global_rx_noalloc(None, 0, 0, 0, 0, 0, None, 0, 0.0, 0, None, None, None, -1) == \
        hs.HSAD_E_INVALID


def test_noalloc_after_larger_layout_and_warmup_status(hs):
    """Each region of the shared array is written before it is read: a call on a smaller
    cube (fewer lines, fewer bands, a smaller padded band count) after a larger one, and a
    good call after one that stopped at HSAD_E_NOT_READY, both match a fresh CUBE-mode
    context."""
    from gen import PushbroomScene
    big_sc = PushbroomScene(96, 130, seed=33)
    big = big_sc.lines(0, 60).view(np.int16)
    small_sc = PushbroomScene(64, 40, seed=34)
    small = small_sc.lines(0, 20).view(np.int16)
    rc, s_big, _ = _noalloc(hs, big, "u16", "fp32", big_sc.gain, "abs", 0.0, 0)
    assert rc == hs.HSAD_OK
    rc0, s0, m0 = _context_scores(hs, small, "u16", "fp32", small_sc.gain, "abs", 0.0, 0)
    assert rc0 == hs.HSAD_OK
    tau = 40 + 6 * np.sqrt(80)
    rc, s, m = _noalloc(hs, small, "u16", "fp32", small_sc.gain, "abs", 0.0, 0)
    assert rc == hs.HSAD_OK
    assert rel_err(s, s0)[0] <= TOL["fp32"] and mask_mismatch(m, s0, tau, MARGIN["fp32"]) == 0
    # 8 pixels of 40 bands: fewer than B + 1, nothing to score
    rc, s_nr, m_nr = _noalloc(hs, np.ascontiguousarray(small[:1, :8]), "u16", "bf16", small_sc.gain, "abs", 0.0, 0)
    assert rc == hs.HSAD_E_NOT_READY and np.isnan(s_nr).all() and (m_nr == 0).all()
    rc, s, m = _noalloc(hs, small, "u16", "fp32", small_sc.gain, "abs", 0.0, 0)
    assert rc == hs.HSAD_OK
    assert rel_err(s, s0)[0] <= TOL["fp32"] and mask_mismatch(m, s0, tau, MARGIN["fp32"]) == 0
