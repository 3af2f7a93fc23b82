"""The covariance sums of uint16 input are integer work: bit-exact against NumPy int64.

Sec. 3.3 builds mu and Sigma from per-band sums over the pixels; with x' = DN - c an
integer, S1 = sum x' and S2 = sum x' x'^T are exact integers. The tensor-core SYRK
(integer split into BF16 halves, FP32 accumulation bounded to 4096 pixels, FP64
combination) must reproduce them exactly, including the sliced path for lines wider
than 4096 pixels and the cube path.
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


def _exact(lines):
    """Shift, S1, S2 of all lines with the shift taken from line 0 (int64, exact)."""
    x0 = lines[0].astype(np.int64)
    W = x0.shape[0]
    c = np.rint(x0.sum(axis=0) / W).astype(np.int64)
    X = lines.reshape(-1, lines.shape[-1]).astype(np.int64) - c
    return c, X.sum(axis=0), X.T @ X


@pytest.mark.parametrize("T,W,B,mode", [
    (12, 96, 40, "exclusive"), (9, 700, 270, "inclusive"), (5, 130, 129, "exclusive"),
    (3, 5000, 64, "exclusive"), (4, 33, 448, "exclusive"),
])
def test_stream_sums_bit_exact(hs, T, W, B, mode):
    from gen import PushbroomScene
    lines = PushbroomScene(W, B, seed=T * 7 + B).lines(0, T)
    det = hs.Detector(width=W, bands=B, stats_mode=mode, max_batch_lines=4)
    det.push(lines)
    rc, n, c, s1, s2 = hs.hsad_get_stats(det.ctx, B)
    det.close()
    assert rc == hs.HSAD_OK and n == T * W
    ce, s1e, s2e = _exact(lines)
    np.testing.assert_array_equal(c, ce.astype(np.float64))
    np.testing.assert_array_equal(s1, s1e.astype(np.float64))
    lo = np.tril_indices(B)
    np.testing.assert_array_equal(s2[lo], s2e[lo].astype(np.float64))


def test_cube_sums_bit_exact(hs):
    from gen import PushbroomScene
    lines = PushbroomScene(300, 200, seed=99).lines(0, 30)
    det = hs.Detector(width=300, bands=200, stats_mode="cube", cube_lines=16)
    det.push(lines)            # one full cube (16 lines) + 14 lines pending
    det.flush()                # the partial cube of 14 lines is scored
    rc, n, c, s1, s2 = hs.hsad_get_stats(det.ctx, 200)
    det.close()
    assert rc == hs.HSAD_OK and n == 14 * 300
    ce, s1e, s2e = _exact(lines[16:])
    np.testing.assert_array_equal(c, ce.astype(np.float64))
    np.testing.assert_array_equal(s1, s1e.astype(np.float64))
    lo = np.tril_indices(200)
    np.testing.assert_array_equal(s2[lo], s2e[lo].astype(np.float64))
