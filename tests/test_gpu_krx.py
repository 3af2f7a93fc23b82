"""Subsampled kernel RX on the GPU against the FP64 oracle (needs a GB300).

Every call goes through the C ABI (hsad_krx). Cases span several 32-pixel CTAs with a
ragged tail, background sizes from 2 to the 512 maximum (multiples and non-multiples of
the 64-sample chunks and 256-output passes), odd and large band counts, float and uint16
input, per-band gains, both threshold forms and a given kernel width. Tolerance: the FP32
path's 1e-4 relative error of the RX scores (the per-pixel steps whose rounding the
ridge-regularised inverse amplifies carry float-float sums); masks bit-exact outside the
margin.
"""
import numpy as np
import pytest

from oracle import krx
from tests._parity import MARGIN, TOL, mask_mismatch, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_13509_gb300 as hs
    return hs


def _gpu(hs, cube, idx, dtype="u16", c=0.0, eps=1e-2, gain=None, mode="abs", tau=0.0, flags=0):
    import torch
    B = cube.shape[-1]
    flat = np.ascontiguousarray(cube.reshape(-1, B))
    n = flat.shape[0]
    x = torch.from_numpy(flat.view(np.int16) if dtype == "u16" else flat).cuda()
    s = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
    m = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
    rc = hs.hsad_krx(x, n, B, hs.HSAD_U16 if dtype == "u16" else hs.HSAD_F32, idx, c, eps, gain,
                     hs.HSAD_REL if mode == "rel" else hs.HSAD_ABS, tau, flags, s, m, None, 0)
    torch.cuda.synchronize()
    return rc, s.cpu().numpy(), m.cpu().numpy()


def _scene(L, W, B, seed):
    from gen import PushbroomScene
    sc = PushbroomScene(W, B, seed=seed)
    return sc, sc.lines(0, L)


@pytest.mark.parametrize("L,W,B,m", [(8, 100, 64, 256), (6, 61, 33, 2), (6, 61, 33, 3), (10, 96, 130, 100),
                                     (4, 200, 270, 64), (5, 77, 448, 300), (4, 170, 20, 512), (2, 70, 512, 129)])
def test_krx_u16_matches_oracle(hs, L, W, B, m):
    from gen import subsample_indices
    sc, cube = _scene(L, W, B, seed=1000 + B + m)
    idx = subsample_indices(L * W, m, seed=B + m)
    rc, s, mk = _gpu(hs, cube, idx, gain=sc.gain)
    assert rc == hs.HSAD_OK, hs.hsad_status_string(rc)
    ref, _ = krx.subsampled_krx(cube, idx, eps=1e-2, gain=sc.gain, offset=sc.offset)
    ref = ref.ravel()
    emax, _ = rel_err(s, ref)
    assert emax <= TOL["fp32"], emax
    tau = B + 6 * np.sqrt(2 * B)
    assert mask_mismatch(mk, ref, tau, MARGIN["fp32"]) == 0


def test_krx_float_input_given_width_and_rel_threshold(hs):
    from gen import config1_cube, subsample_indices
    cube, anom, _ = config1_cube()
    idx = subsample_indices(cube.shape[0] * cube.shape[1], 256, seed=3)
    c = 1.0  # a given kernel width (the default would be the mean pairwise distance, about 4.2)
    ref, bg = krx.subsampled_krx(cube, idx, c=c, eps=1e-2)
    ref = ref.ravel()
    rc, s, mk = _gpu(hs, cube, idx, dtype="f32", c=c, mode="rel", tau=0.110)
    assert rc == hs.HSAD_OK
    emax, _ = rel_err(s, ref)
    assert emax <= TOL["fp32"], emax
    assert mask_mismatch(mk, ref / ref.max(), 0.110, 2 * MARGIN["fp32"]) == 0
    # normalised scores: delta / max
    rc, s2, _ = _gpu(hs, cube, idx, dtype="f32", c=c, mode="rel", tau=0.110, flags=hs.HSAD_NORMALIZE_SCORES)
    assert rc == hs.HSAD_OK and abs(float(np.max(s2)) - 1.0) < 1e-6
    assert np.max(np.abs(s2 - ref / ref.max())) < 2e-4


@pytest.mark.parametrize("eps", [1e-1, 3e-3])
def test_krx_ridge_values(hs, eps):
    from gen import subsample_indices
    sc, cube = _scene(6, 128, 48, seed=77)
    idx = subsample_indices(6 * 128, 160, seed=9)
    rc, s, _ = _gpu(hs, cube, idx, eps=eps, gain=sc.gain)
    assert rc == hs.HSAD_OK
    ref, _ = krx.subsampled_krx(cube, idx, eps=eps, gain=sc.gain)
    emax, _ = rel_err(s, ref.ravel())
    assert emax <= TOL["fp32"], emax


def test_krx_in_sample_identity_and_repeat_calls(hs):
    """The background pixels' own scores sum to (m - 1) sum_j l_j^2 / (l_j + lam)^2 over the
    eigenvalues of K~ (computed here from the oracle's Gram matrix); two calls in a row give
    identical scores."""
    from gen import subsample_indices
    sc, cube = _scene(8, 64, 40, seed=5)
    idx = subsample_indices(8 * 64, 96, seed=5)
    rc, s, _ = _gpu(hs, cube, idx, gain=sc.gain)
    rc2, s2, _ = _gpu(hs, cube, idx, gain=sc.gain)
    assert rc == rc2 == hs.HSAD_OK
    np.testing.assert_array_equal(s, s2)
    _, bg = krx.subsampled_krx(cube, idx, eps=1e-2, gain=sc.gain)
    lj = np.linalg.eigvalsh(bg["Kc"])
    ident = (bg["m"] - 1) * float((lj ** 2 / (lj + bg["lam"]) ** 2).sum())
    assert abs(float(s[idx].astype(np.float64).sum()) - ident) <= 1e-4 * ident


def test_krx_rejections(hs):
    import torch
    x = torch.zeros((100, 8), dtype=torch.int16, device="cuda")
    s = torch.zeros(100, dtype=torch.float32, device="cuda")
    m = torch.zeros(100, dtype=torch.uint8, device="cuda")

    def call(idx, n=100, B=8, eps=1e-2, c=0.0, dtype=None, flags=0):
        return hs.hsad_krx(x, n, B, hs.HSAD_U16 if dtype is None else dtype, idx, c, eps, None, hs.HSAD_ABS,
                           0.0, flags, s, m, None, 0)
    assert call([1, 1, 2]) == hs.HSAD_E_INVALID              # repeated index
    assert call([0, 100]) == hs.HSAD_E_INVALID               # out of range
    assert call([5]) == hs.HSAD_E_INVALID                    # m < 2
    assert call(list(range(513)), n=600) == hs.HSAD_E_INVALID  # m > 512
    assert call([0, 1], eps=0.0) == hs.HSAD_E_INVALID
    assert call([0, 1], c=-1.0) == hs.HSAD_E_INVALID
    assert call([0, 1], B=513) == hs.HSAD_E_INVALID
    assert call([0, 1], dtype=9) == hs.HSAD_E_INVALID
    assert call([0, 1], flags=4) == hs.HSAD_E_INVALID
    xf = torch.zeros((100, 8), dtype=torch.float32, device="cuda")
    xf[3, 2] = float("nan")
    assert hs.hsad_krx(xf, 100, 8, hs.HSAD_F32, [0, 1, 2], 0.0, 1e-2, None, hs.HSAD_ABS, 0.0, 0, s, m, None,
                       0) == hs.HSAD_E_INVALID_DATA


def test_krx_anomalies_rank_high(hs):
    """Implanted anomalies of the float mixture cube rank above the background (Sec. 2.2's
    comparison is of detection quality; here only the ranking property is required)."""
    from gen import config1_cube, subsample_indices
    cube, anom, _ = config1_cube()
    idx = subsample_indices(cube.shape[0] * cube.shape[1], 256, seed=11)
    rc, s, _ = _gpu(hs, cube, idx, dtype="f32")
    assert rc == hs.HSAD_OK
    s = s.reshape(anom.shape)
    assert np.median(s[anom]) > np.percentile(s[~anom], 90)
