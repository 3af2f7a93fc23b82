"""Full-size workloads in the launch configuration bench.py times, checked on sampled lines.

640 px x 270 bands x 4000 lines (whole stream in one batch) and 1024 px x 448 bands x
8000 lines (batches of 2000), EXCLUSIVE statistics. The oracle scores sampled lines one
by one against all the lines before them: at least one in every batch, the first lines of
later batches (scored with the factor carried over the batch boundary) and the last line. Tolerances as everywhere:
relative error <= 1e-4 (FP32), <= 1e-2 (BF16 / FP16); masks bit-exact outside the margin.

With HSAD_PRECISION_REPORT=<file> the per-precision error report (against the oracle and
against the FP32 path, and the condition number of the last sampled line's covariance)
is written there as JSON.
"""
import json
import os

import numpy as np
import pytest

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


def _run(hs, lines, sc, prec, batch):
    import torch
    T, W, B = lines.shape
    x = torch.from_numpy(lines.view(np.int16)).cuda()
    s = torch.empty((T, W), dtype=torch.float32, device="cuda")
    m = torch.empty((T, W), dtype=torch.uint8, device="cuda")
    det = hs.Detector(width=W, bands=B, stats_mode="exclusive", precision=prec, gain=sc.gain, offset=sc.offset,
                      max_batch_lines=batch, result_lines=T)
    rc, first = hs.hsad_push_lines(det.ctx, x, T, hs.HSAD_DEVICE)
    assert rc == hs.HSAD_OK
    rc = hs.hsad_scores(det.ctx, first, T, s, m, hs.HSAD_DEVICE, -1)
    assert rc in (hs.HSAD_OK, hs.HSAD_E_NOT_READY)
    st = np.empty(T, np.int32)
    assert hs.hsad_line_status(det.ctx, first, T, st, 0) == hs.HSAD_OK
    det.close()
    return s.cpu().numpy(), m.cpu().numpy(), st


@pytest.fixture(scope="module")
def stream_640x270():
    from gen import config_scene
    sc, T = config_scene("stream_640x270")
    return sc, sc.lines(0, T)


@pytest.fixture(scope="module")
def stream_1024x448():
    from gen import config_scene
    sc, T = config_scene("precision_1024x448")
    return sc, sc.lines(0, T)


_REF = {}      # (workload, line) -> oracle scores, shared by the precisions
_RESULTS = {}  # (workload, precision) -> (scores, mask) of the sampled lines
_REPORT = {}


def _write_report():
    path = os.environ.get("HSAD_PRECISION_REPORT")
    if path:
        with open(path, "w") as f:
            json.dump(_REPORT, f, indent=1, sort_keys=True)


def _check(s, m, st, lines, sc, prec, sample, name):
    T, W, B = lines.shape
    # warm-up: line t is ready once t * W >= B + 1 pixels precede it
    first_ready = -(-(B + 1) // W)
    assert (st[:first_ready] == orx.NOT_READY).all() and (st[first_ready:] == orx.OK).all()
    assert np.isnan(s[:first_ready]).all() and np.isfinite(s[first_ready:]).all()
    tau = B + 6 * np.sqrt(2 * B)
    rep = {"lines": sample, "max_rel_err": 0.0, "p999_rel_err": 0.0, "mask_diff_outside_margin": 0,
           "mask_diff_total": 0, "pixels": 0}
    for t in sample:
        key = (name, t)
        if key not in _REF:
            ref, rst = orx.stream_rx_line(lines, t, "exclusive", gain=sc.gain, offset=sc.offset, n_lines=T)
            assert rst == orx.OK
            _REF[key] = ref
        ref = _REF[key]
        emax, e999 = rel_err(s[t], ref)
        assert emax <= TOL[prec], (t, emax)
        bad = mask_mismatch(m[t], ref, tau, MARGIN[prec])
        assert bad == 0, t
        rep["max_rel_err"] = max(rep["max_rel_err"], emax)
        rep["p999_rel_err"] = max(rep["p999_rel_err"], e999)
        rep["mask_diff_outside_margin"] += bad
        rep["mask_diff_total"] += int((m[t].astype(bool) != (ref > tau)).sum())
        rep["pixels"] += W
    _RESULTS[(name, prec)] = (s[sample].copy(), m[sample].copy())
    fp32 = _RESULTS.get((name, "fp32"))
    if fp32 is not None:  # every precision run so far against the FP32 path
        for (n2, p2), (s2, m2) in _RESULTS.items():
            if n2 == name and p2 != "fp32":
                e = np.abs(s2.astype(np.float64) - fp32[0]) / np.maximum(fp32[0], 1.0)
                _REPORT[f"{name}/{p2}"]["vs_fp32_max_rel"] = float(e.max())
                _REPORT[f"{name}/{p2}"]["vs_fp32_mask_diff"] = int((m2 != fp32[1]).sum())
        a, b = orx.statistics_lines(sample[-1], "exclusive", 0, T)
        _, cov, _ = orx._stats_over_lines(lines, a, b, sc.gain, sc.offset, 256)
        ev = np.linalg.eigvalsh(cov)
        rep["kappa_sigma_last_sample"] = float(ev[-1] / ev[0])
    _REPORT[f"{name}/{prec}"] = rep
    _write_report()


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_stream_640x270_full(hs, stream_640x270, prec):
    sc, lines = stream_640x270
    s, m, st = _run(hs, lines, sc, prec, 4000)
    _check(s, m, st, lines, sc, prec, sample=[1, 2, 500, 1999, 3000, 3999], name="stream_640x270")


@pytest.mark.parametrize("prec", ["bf16", "fp16", "fp32"])
def test_stream_1024x448_full(hs, stream_1024x448, prec):
    sc, lines = stream_1024x448
    s, m, st = _run(hs, lines, sc, prec, 2000)
    # one line in each of the four 2000-line batches, the first line of every batch after
    # the first (scored with the factor carried across the batch boundary) and the last line
    _check(s, m, st, lines, sc, prec, sample=[1, 2001, 2400, 4001, 6001, 7999], name="precision_1024x448")
