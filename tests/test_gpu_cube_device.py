"""Global RX of device-generated cubes of stress-workload shape (CUBE mode, zero-copy push).

Two cubes cut from the stress workload's range (500 lines x 2048 px x 224 bands, 0.46 GB,
and 200 lines x 2048 px x 448 bands, the largest band count, 0.37 GB) are drawn on the
GPU, scored in place, and compared with the FP64 oracle on every pixel. Independently of the oracle,
the in-sample scores must obey the exact identity mean(delta) = B (N-1) / N and the
leverage bound delta <= (N-1)^2 / N (Sec. 3.3 statistics over all pixels of the cube).
"""
import numpy as np
import pytest

import oracle
from tests._parity import MARGIN, TOL, mask_mismatch, rel_err

pytestmark = pytest.mark.gpu

SHAPES = [(500, 2048, 224), (200, 2048, 448)]


@pytest.fixture(scope="module")
def hs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_13509_gb300 as hs
    return hs


@pytest.fixture(scope="module", params=SHAPES, ids=lambda s: "x".join(map(str, s)))
def cube(request):
    import torch
    from gen import PushbroomScene
    from gen.device import DeviceScene
    L, W, B = request.param
    sc = PushbroomScene(W, B, seed=77 + B)
    x = torch.empty((L, W, B), dtype=torch.int16, device="cuda")
    DeviceScene(sc).generate(x, 0, seed=77 + B)
    torch.cuda.synchronize()
    host = x.cpu().numpy().view(np.uint16)
    assert host.max() <= 4095 and host.min() >= 0
    ref, _ = oracle.global_rx(host, sc.gain, sc.offset)
    yield sc, x, ref
    del x
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_device_cube_matches_oracle_and_identity(hs, cube, prec):
    import torch
    sc, x, ref = cube
    L, W, B = x.shape
    s = torch.empty((L, W), dtype=torch.float32, device="cuda")
    m = torch.empty((L, W), dtype=torch.uint8, device="cuda")
    det = hs.Detector(width=W, bands=B, stats_mode="cube", cube_lines=L, precision=prec, gain=sc.gain,
                      offset=sc.offset, result_lines=L)
    rc, first = hs.hsad_push_lines(det.ctx, x, L, hs.HSAD_DEVICE)
    assert rc == hs.HSAD_OK
    assert hs.hsad_scores(det.ctx, first, L, s, m, hs.HSAD_DEVICE, -1) == hs.HSAD_OK
    det.close()
    d = s.cpu().numpy()
    emax, _ = rel_err(d, ref)
    assert emax <= TOL[prec], emax
    tau = B + 6 * np.sqrt(2 * B)
    assert mask_mismatch(m.cpu().numpy(), ref, tau, MARGIN[prec]) == 0
    N = L * W
    mean = d.astype(np.float64).mean()
    assert abs(mean - B * (N - 1) / N) / B < (1e-5 if prec == "fp32" else 2e-3)
    assert d.max() <= (N - 1) ** 2 / N
