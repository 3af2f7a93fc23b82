"""CUDA path vs the FP64 oracle on seeded inputs (needs a GB300).

Every call goes through the C ABI (via the ctypes binding). Sizes span several
64-wide tiles with ragged tails; the edge cases cover B = 1..3, W = 1, warm-up,
statistics resets, partial cubes and a non positive definite covariance.
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


def _scene_lines(T, W, B, seed):
    from gen import PushbroomScene
    sc = PushbroomScene(W, B, seed=seed)
    return sc, sc.lines(0, T)


def _run(hs, lines, **kw):
    det = hs.Detector(width=lines.shape[1], bands=lines.shape[2], **kw)
    first = det.push(lines)
    if kw.get("stats_mode") == "cube":
        det.flush()
    rc, s, m, st = det.scores(first, lines.shape[0])
    launches = det.kernel_launches
    det.close()
    return rc, s, m, st, launches


# ------------------------------------------------------------------ global RX (cube mode)
@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_config1_cube_global_rx(hs, prec):
    """64 x 128 x 64 float32 mixture cube, global RX, REL threshold 0.110 (Sec. 3.3)."""
    from gen import config1_cube
    cube, anom, _ = config1_cube()
    dref, dnorm = oracle.global_rx(cube)
    rc, s, m, st, nl = _run(hs, cube, in_dtype="f32", precision=prec, stats_mode="cube", cube_lines=64,
                            threshold_mode="rel", threshold=0.110)
    assert rc == hs.HSAD_OK and (st == 0).all() and nl > 0
    # float input: the centred values are split into two BF16 (or two FP16) terms, 16 (22)
    # of their 24 bits, and G into hi + lo; the scores still meet each precision's tolerance
    emax, _ = rel_err(s, dref)
    assert emax <= TOL[prec], emax
    assert mask_mismatch(m, dnorm, 0.110, 2 * MARGIN[prec]) == 0
    assert np.median(s[anom]) > np.percentile(s[~anom], 99)


def test_config1_normalized_scores(hs):
    from gen import config1_cube
    cube, _, _ = config1_cube()
    _, dnorm = oracle.global_rx(cube)
    rc, s, m, st, _ = _run(hs, cube, in_dtype="f32", stats_mode="cube", cube_lines=64, threshold_mode="rel",
                           threshold=0.110, flags=hs.HSAD_NORMALIZE_SCORES)
    assert rc == hs.HSAD_OK
    assert abs(np.nanmax(s) - 1.0) < 1e-6
    assert np.max(np.abs(s - dnorm)) < 2e-4


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_cube_mode_u16_with_partial_cube(hs, prec):
    sc, lines = _scene_lines(52, 70, 33, seed=7)   # two cubes of 20 lines + a partial of 12
    rc, s, m, st, _ = _run(hs, lines, stats_mode="cube", cube_lines=20, precision=prec,
                           gain=sc.gain, offset=sc.offset)
    assert rc == hs.HSAD_OK
    ref, _ = orx.stream_rx(lines, oracle.CUBE, cube_lines=20, gain=sc.gain, offset=sc.offset)
    emax, _ = rel_err(s, ref)
    assert emax <= TOL[prec], emax
    tau = 33 + 6 * np.sqrt(66)
    assert mask_mismatch(m, ref, tau, MARGIN[prec]) == 0


# ------------------------------------------------------------------ streamed forms
@pytest.mark.parametrize("mode", ["exclusive", "inclusive"])
@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_stream_modes_small(hs, mode, prec):
    sc, lines = _scene_lines(40, 96, 24, seed=3)
    rc, s, m, st, _ = _run(hs, lines, stats_mode=mode, precision=prec, gain=sc.gain, offset=sc.offset,
                           max_batch_lines=16)
    ref, rst = orx.stream_rx(lines, getattr(oracle, mode.upper()), gain=sc.gain, offset=sc.offset)
    assert rc in (hs.HSAD_OK, hs.HSAD_E_NOT_READY)
    np.testing.assert_array_equal(st, rst)
    emax, _ = rel_err(s, ref)
    assert emax <= TOL[prec], emax
    tau = 24 + 6 * np.sqrt(48)
    assert mask_mismatch(m, ref, tau, MARGIN[prec]) == 0


@pytest.mark.parametrize("W,B", [(1, 1), (7, 1), (3, 2), (9, 3), (65, 64), (33, 127), (64, 128),
                                 (17, 129), (130, 200), (130, 448), (40, 512)])
def test_stream_ragged_shapes(hs, W, B):
    sc, lines = _scene_lines(max(6, (B + 1) // W + 4), W, B, seed=W * 1000 + B)
    rc, s, m, st, _ = _run(hs, lines, stats_mode="exclusive", gain=sc.gain, offset=sc.offset)
    ref, rst = orx.stream_rx(lines, oracle.EXCLUSIVE, gain=sc.gain, offset=sc.offset)
    np.testing.assert_array_equal(st, rst)
    emax, _ = rel_err(s, ref)
    assert emax <= TOL["fp32"], emax


@pytest.mark.parametrize("W,B,mode", [(70, 200, "exclusive"), (33, 270, "inclusive"), (9, 448, "exclusive")])
def test_float_stream_tensor_core_factor_simt_solve(hs, W, B, mode):
    """Float input at B >= 192: the tensor-core factor with the FP32 solve on the SIMT cores
    (the transposed FP32 operand), against the oracle at the FP32 tolerance."""
    from gen import IllConditionedScene
    T = max(6, (B + 1) // W + 4)
    lines = IllConditionedScene(W, B, seed=W * 7 + B, decades=2.0, dtype="f32").lines(0, T)  # kappa 1e4
    rc, s, m, st, _ = _run(hs, lines, in_dtype="f32", stats_mode=mode)
    ref, rst = orx.stream_rx(lines, oracle.EXCLUSIVE if mode == "exclusive" else oracle.INCLUSIVE)
    np.testing.assert_array_equal(st, rst)
    emax, _ = rel_err(s, ref)
    assert emax <= TOL["fp32"], emax


@pytest.mark.parametrize("W,B", [(1, 1), (7, 3), (129, 64), (65, 65), (33, 127), (300, 130), (130, 270),
                                 (640, 270), (130, 448), (40, 500), (21, 512)])
def test_stream_bf16_ragged_shapes(hs, W, B):
    """BF16 streams of uint16 lines whiten by the blocked triangular solve: one and several
    64-band blocks with ragged tails, odd B (2-byte raw loads), ring depths from 1 to 9
    stages, B up to the 512-band maximum."""
    sc, lines = _scene_lines(max(6, (B + 1) // W + 4), W, B, seed=W * 1000 + B + 1)
    rc, s, m, st, _ = _run(hs, lines, stats_mode="exclusive", precision="bf16", gain=sc.gain, offset=sc.offset)
    ref, rst = orx.stream_rx(lines, oracle.EXCLUSIVE, gain=sc.gain, offset=sc.offset)
    np.testing.assert_array_equal(st, rst)
    emax, _ = rel_err(s, ref)
    assert emax <= TOL["bf16"], emax
    tau = B + 6 * np.sqrt(2 * B)
    assert mask_mismatch(m, ref, tau, MARGIN["bf16"]) == 0


@pytest.mark.parametrize("prec,dtype,B,mode,form,tcw", [("bf16", "u16", 270, "exclusive", 1, True),
                                                         ("bf16", "u16", 448, "inclusive", 1, True),
                                                         ("bf16", "u16", 512, "exclusive", 1, True),
                                                         ("bf16", "f32", 270, "exclusive", 0, True),
                                                         ("bf16", "u16", 270, "cube", 0, True),
                                                         ("fp16", "u16", 270, "exclusive", 0, True),
                                                         ("fp32", "u16", 270, "exclusive", 1, True),
                                                         ("fp32", "u16", 128, "exclusive", 1, False),
                                                         ("fp32", "f32", 270, "inclusive", 1, False),
                                                         ("fp32", "u16", 512, "exclusive", 1, True),
                                                         ("fp32", "f32", 270, "cube", 0, False)])
def test_whitening_form_per_context(hs, prec, dtype, B, mode, form, tcw):
    """Form (triangular solve or explicit inverse) and units (tensor or SIMT cores) of each
    context kind: FP32 on the tensor cores needs uint16 input, streamed statistics and
    B >= 192 (the tensor-core factor)."""
    kw = dict(cube_lines=16) if mode == "cube" else {}
    det = hs.Detector(width=32, bands=B, precision=prec, in_dtype=dtype, stats_mode=mode, **kw)
    assert det.whitening_form == form
    assert det.whitening_tensor_cores == tcw
    det.close()
    if prec == "fp32" and dtype == "u16" and mode != "cube":  # the FP64 factor keeps the SIMT solve
        det = hs.Detector(width=32, bands=B, precision=prec, in_dtype=dtype, stats_mode=mode,
                          factor_precision=hs.HSAD_FACTOR_FP64)
        assert det.whitening_form == 1 and not det.whitening_tensor_cores
        det.close()
    # HSAD_FORCE_INVERSE keeps the explicit inverse everywhere
    det = hs.Detector(width=32, bands=B, precision=prec, in_dtype=dtype, stats_mode=mode,
                      flags=hs.HSAD_FORCE_INVERSE, **kw)
    assert det.whitening_form == hs.HSAD_FORM_INVERSE
    det.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_forced_inverse_form_matches_oracle(hs, prec):
    """A streamed context forced to the explicit-inverse form (full L^{-1}, one GEMM) scores
    the same lines as the oracle within each precision's tolerance."""
    sc, lines = _scene_lines(30, 130, 200, seed=31)
    rc, s, m, st, _ = _run(hs, lines, stats_mode="exclusive", precision=prec, gain=sc.gain, offset=sc.offset,
                           flags=hs.HSAD_FORCE_INVERSE, max_batch_lines=11)
    ref, rst = orx.stream_rx(lines, oracle.EXCLUSIVE, gain=sc.gain, offset=sc.offset)
    np.testing.assert_array_equal(st, rst)
    emax, _ = rel_err(s, ref)
    assert emax <= TOL[prec], emax
    assert mask_mismatch(m, ref, 200 + 6 * np.sqrt(400), MARGIN[prec]) == 0


# ------------------------------------------------------------------ FP64 factor form
@pytest.mark.parametrize("prec,mode,W,B,batch", [("fp32", "exclusive", 33, 127, 0), ("fp32", "exclusive", 130, 270, 1),
                                                 ("fp32", "inclusive", 130, 448, 5), ("bf16", "exclusive", 300, 130, 0),
                                                 ("bf16", "exclusive", 130, 270, 1), ("fp16", "exclusive", 65, 65, 0),
                                                 ("fp32", "cube", 64, 100, 0), ("bf16", "cube", 64, 100, 0)])
def test_fp64_factor_matches_oracle(hs, prec, mode, W, B, batch):
    """factor_precision = HSAD_FACTOR_FP64: the factor's O(B^3) work in FP64 instead of
    float-float, in one-CTA (whole pushes) and cluster (one-line pushes) launch shapes, in
    both whitening forms; same tolerances, and the scores differ from the float-float
    factor's only in the last bits."""
    T = max(8, (B + 1) // W + 5)
    sc, lines = _scene_lines(T, W, B, seed=W * 7 + B)
    kw = dict(stats_mode=mode, precision=prec, gain=sc.gain, offset=sc.offset)
    if mode == "cube":
        kw["cube_lines"] = T
    out = {}
    for fp in ("fp64", "ff"):
        det = hs.Detector(width=W, bands=B, factor_precision=fp, **kw)
        if batch:
            for t in range(0, T, batch):
                det.push(lines[t:t + batch])
        else:
            det.push(lines)
        if mode == "cube":
            det.flush()
        rc, s, m, st = det.scores(0, T)
        det.close()
        out[fp] = (s, m, st)
    if mode == "cube":
        ref, rst = orx.stream_rx(lines, oracle.CUBE, cube_lines=T, gain=sc.gain, offset=sc.offset)
    else:
        ref, rst = orx.stream_rx(lines, getattr(oracle, mode.upper()), gain=sc.gain, offset=sc.offset)
    s, m, st = out["fp64"]
    np.testing.assert_array_equal(st, rst)
    emax, _ = rel_err(s, ref)
    assert emax <= TOL[prec], emax
    assert mask_mismatch(m, ref, B + 6 * np.sqrt(2 * B), MARGIN[prec]) == 0
    ok = np.isfinite(ref)
    d = np.abs(out["ff"][0][ok].astype(np.float64) - s[ok]) / np.maximum(ref[ok], 1.0)
    assert d.max() <= (1e-5 if prec == "fp32" else 1e-3), d.max()


def test_stream_resets_and_warmup(hs):
    sc, lines = _scene_lines(50, 40, 20, seed=11)
    kw = dict(stats_mode="exclusive", cube_lines=16, warmup_pixels=100, gain=sc.gain, offset=sc.offset,
              max_batch_lines=7)
    rc, s, m, st, _ = _run(hs, lines, **kw)
    ref, rst = orx.stream_rx(lines, oracle.EXCLUSIVE, cube_lines=16, warmup_pixels=100, gain=sc.gain,
                             offset=sc.offset)
    np.testing.assert_array_equal(st, rst)
    assert (rst == orx.NOT_READY).sum() >= 9     # 3 lines after each reset
    emax, _ = rel_err(s, ref)
    assert emax <= TOL["fp32"], emax


def test_host_and_device_push_agree(hs):
    import torch
    sc, lines = _scene_lines(30, 64, 32, seed=5)
    a = _run(hs, lines, stats_mode="exclusive")
    det = hs.Detector(width=64, bands=32, stats_mode="exclusive")
    first = det.push(torch.from_numpy(lines.view(np.int16)).cuda())   # same bytes as uint16
    rc, s, m, st = det.scores(first, 30)
    det.close()
    np.testing.assert_array_equal(np.isnan(a[1]), np.isnan(s))
    np.testing.assert_array_equal(np.nan_to_num(a[1]), np.nan_to_num(s))
    np.testing.assert_array_equal(a[2], m)


def test_pushes_of_one_line_match_one_batch(hs):
    sc, lines = _scene_lines(24, 48, 16, seed=9)
    a = _run(hs, lines, stats_mode="exclusive")
    det = hs.Detector(width=48, bands=16, stats_mode="exclusive")
    ids = [det.push(lines[t:t + 1]) for t in range(24)]
    assert ids == list(range(24))
    rc, s, m, st = det.scores(0, 24)
    det.close()
    np.testing.assert_allclose(np.nan_to_num(s), np.nan_to_num(a[1]), rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("B", [16, 130])
def test_cluster_and_single_cta_factors_agree_bitwise(hs, B):
    """One 160-line push factors each line in one CTA; pushes of one line spread each
    factorisation over a thread-block cluster. The covariance sums are exact and both
    factor forms perform the same FP64 operations in the same order per element, so the
    scores must be identical, not merely close."""
    sc, lines = _scene_lines(160, 40, B, seed=12)
    a = _run(hs, lines, stats_mode="exclusive", precision="fp32")
    det = hs.Detector(width=40, bands=B, stats_mode="exclusive", precision="fp32")
    for t in range(160):
        det.push(lines[t:t + 1])
    rc, s, m, st = det.scores(0, 160)
    det.close()
    np.testing.assert_array_equal(s, a[1])
    np.testing.assert_array_equal(m, a[2])


@pytest.mark.parametrize("prec,B", [("fp32", 270), ("bf16", 448), ("fp32", 192)])
def test_tensor_core_factor_is_batch_invariant(hs, prec, B):
    """From B = 192 the streamed factor runs on the tensor cores (64-column panels, exact
    digit-split trailing updates); each line's factor is computed the same way whatever the
    batch holds, so one-line pushes, uneven pushes and one whole push give identical scores,
    and they match the oracle."""
    sc, lines = _scene_lines(24, 64, B, seed=B + 3)
    a = _run(hs, lines, stats_mode="exclusive", precision=prec, gain=sc.gain, offset=sc.offset)
    outs = []
    for chunks in ([1] * 24, [5, 1, 7, 2, 9]):
        det = hs.Detector(width=64, bands=B, stats_mode="exclusive", precision=prec, gain=sc.gain,
                          offset=sc.offset)
        t = 0
        for n in chunks:
            det.push(lines[t:t + n])
            t += n
        rc, s, m, st = det.scores(0, 24)
        det.close()
        outs.append((s, m))
    for s, m in outs:
        np.testing.assert_array_equal(s, a[1])
        np.testing.assert_array_equal(m, a[2])
    ref, rst = orx.stream_rx(lines, oracle.EXCLUSIVE, gain=sc.gain, offset=sc.offset)
    np.testing.assert_array_equal(a[3], rst)
    emax, _ = rel_err(a[1], ref)
    assert emax <= TOL[prec], emax


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_cuda_graph_replay_matches_direct_launches(hs, prec):
    """HSAD_CUDA_GRAPHS replays a captured launch sequence per batch size; the kernels and
    their arguments are those of the direct path, so the scores must be identical."""
    sc, lines = _scene_lines(90, 72, 40, seed=13)
    out = []
    for flags in (0, hs.HSAD_CUDA_GRAPHS):
        det = hs.Detector(width=72, bands=40, stats_mode="exclusive", precision=prec, flags=flags)
        t = 0
        # repeated batch sizes: captured once, replayed; batches above 8 lines launch directly
        for n in [1, 1, 2, 1, 3, 3, 1, 2, 12] * 10:
            if t + n > 90:
                break
            det.push(lines[t:t + n])
            t += n
        rc, s, m, st = det.scores(0, t)
        launches = det.kernel_launches
        det.close()
        out.append((s, m, st, launches))
    np.testing.assert_array_equal(out[1][0], out[0][0])
    np.testing.assert_array_equal(out[1][1], out[0][1])
    np.testing.assert_array_equal(out[1][2], out[0][2])
    assert out[1][3] >= out[0][3]  # every replayed kernel is counted (plus one descriptor write per batch)


def test_autotuned_factor_shapes_give_identical_scores(hs):
    """The autotuner only picks launch shapes; every shape computes the same factor."""
    sc, lines = _scene_lines(40, 48, 24, seed=14)

    def run():
        det = hs.Detector(width=48, bands=24, stats_mode="exclusive", precision="bf16")
        for t in range(0, 40, 2):
            det.push(lines[t:t + 2])
        rc, s, m, st = det.scores(0, 40)
        det.close()
        return s, m

    before = run()
    rc, rows = hs.hsad_autotune_factor(0, 24, "bf16", 8)
    assert rc == hs.HSAD_OK and [int(r[0]) for r in rows] == [1, 2, 4, 8]
    for bucket, cl, ft, ms in rows:
        assert int(cl) in (1, 2, 4, 8, 16) and int(ft) in (96, 128, 256) and ms > 0
    after = run()
    np.testing.assert_array_equal(after[0], before[0])
    np.testing.assert_array_equal(after[1], before[1])
    assert hs.hsad_autotune_factor(0, 24, "bf16", 5000)[0] == hs.HSAD_E_INVALID


@pytest.mark.parametrize("graphs", [False, True])
def test_pinned_pageable_and_device_pushes_agree(hs, graphs):
    """Pinned host lines go to the device by DMA on a copy stream, pageable ones through
    library staging, device lines in place: the scores must be identical, and a pinned
    buffer may be overwritten as soon as its push returns."""
    import torch
    sc, lines = _scene_lines(36, 40, 20, seed=15)
    flags = hs.HSAD_CUDA_GRAPHS if graphs else 0
    chunks = [(0, 1), (1, 7), (8, 1), (9, 1), (10, 7), (17, 7), (24, 12)]

    def run(kind):
        det = hs.Detector(width=40, bands=20, stats_mode="exclusive", precision="bf16", flags=flags)
        buf = torch.empty((12, 40, 20), dtype=torch.int16).pin_memory()
        dev = torch.from_numpy(lines.view(np.int16)).cuda()
        for a, n in chunks:
            if kind == "pageable":
                rc, _ = hs.hsad_push_lines(det.ctx, np.ascontiguousarray(lines[a:a + n]), n, hs.HSAD_HOST)
            elif kind == "pinned":
                buf[:n].copy_(torch.from_numpy(lines[a:a + n].view(np.int16)))
                rc, _ = hs.hsad_push_lines(det.ctx, buf[:n], n, hs.HSAD_HOST)
                buf.fill_(-1)  # reused at once: the push has already copied it
            else:
                rc, _ = hs.hsad_push_lines(det.ctx, dev[a:a + n], n, hs.HSAD_DEVICE)
            assert rc == hs.HSAD_OK
        rc, s, m, st = det.scores(0, 36)
        det.close()
        return s, m

    ref = run("pageable")
    for kind in ("pinned", "device"):
        s, m = run(kind)
        np.testing.assert_array_equal(s, ref[0])
        np.testing.assert_array_equal(m, ref[1])


@pytest.mark.parametrize("mode", ["exclusive", "inclusive"])
def test_statistics_export_import_resumes_bitwise(hs, mode):
    """Checkpoint / resume: a stream exported after 12 lines and imported into a fresh
    context scores the remaining lines exactly as the uninterrupted stream does."""
    sc, lines = _scene_lines(30, 48, 20, seed=16)
    kw = dict(width=48, bands=20, stats_mode=mode, precision="bf16", gain=sc.gain, offset=sc.offset)
    a = hs.Detector(**kw)
    a.push(lines)
    rc, sa, ma, sta = a.scores(0, 30)
    a.close()
    b = hs.Detector(**kw)
    b.push(lines[:12])
    rc, n, shift, s1, s2 = hs.hsad_get_stats(b.ctx, 20)
    b.close()
    assert rc == hs.HSAD_OK and n == 12 * 48
    c = hs.Detector(**kw)
    assert hs.hsad_set_stats(c.ctx, n, shift, s1, s2) == hs.HSAD_OK
    for t in range(12, 30, 6):
        c.push(lines[t:t + 6])
    rc, sc_, mc, stc = c.scores(0, 18)
    assert hs.hsad_set_stats(c.ctx, n, shift, s1, s2) == hs.HSAD_E_INVALID  # context in use
    c.close()
    np.testing.assert_array_equal(sc_, sa[12:])
    np.testing.assert_array_equal(mc, ma[12:])
    np.testing.assert_array_equal(stc, sta[12:])
    cube = hs.Detector(width=48, bands=20, stats_mode="cube", cube_lines=8)
    assert hs.hsad_set_stats(cube.ctx, n, shift, s1, s2) == hs.HSAD_E_INVALID
    bad = np.array(shift, dtype=np.float64)
    bad[0] += 0.5
    d = hs.Detector(**kw)
    assert hs.hsad_set_stats(d.ctx, n, bad, s1, s2) == hs.HSAD_E_INVALID
    cube.close()
    d.close()


def test_large_pinned_push_runs_as_wave_batches_bitwise(hs):
    """A pinned host push of several factor waves runs as a one-wave batch and then whole
    waves, each batch's copy overlapping the previous batch's kernels; the scores equal
    those of the same lines pushed from device memory in one batch."""
    import torch
    T, W, B = 2600, 32, 16
    sc, lines = _scene_lines(T, W, B, seed=17)
    out = []
    for kind in ("pinned", "device"):
        det = hs.Detector(width=W, bands=B, stats_mode="exclusive", precision="bf16", max_batch_lines=4096,
                          result_lines=T)
        if kind == "pinned":
            x = torch.from_numpy(lines.view(np.int16)).pin_memory()
            rc, first = hs.hsad_push_lines(det.ctx, x, T, hs.HSAD_HOST)
        else:
            x = torch.from_numpy(lines.view(np.int16)).cuda()
            rc, first = hs.hsad_push_lines(det.ctx, x, T, hs.HSAD_DEVICE)
        assert rc == hs.HSAD_OK
        rc, s, m, st = det.scores(first, T)
        out.append((s, m, det.kernel_launches))
        det.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])


def test_not_positive_definite_is_reported(hs):
    sc, lines = _scene_lines(12, 40, 8, seed=2)
    lines = lines.copy()
    lines[..., 3] = 1000                          # constant band: singular covariance
    det = hs.Detector(width=40, bands=8, stats_mode="exclusive")
    first = det.push(lines)
    rc, s, m, st = det.scores(first, 12)
    det.close()
    assert rc == hs.HSAD_E_NOT_PD
    assert (st[1:] == hs.LS_NOT_PD).all() and np.isnan(s[1:]).all() and (m == 0).all()


def test_float_push_with_nan_is_rejected(hs):
    x = np.random.default_rng(0).normal(size=(4, 10, 5)).astype(np.float32)
    x[2, 3, 1] = np.nan
    det = hs.Detector(width=10, bands=5, in_dtype="f32", stats_mode="exclusive")
    rc, _ = hs.hsad_push_lines(det.ctx, x, 4, hs.HSAD_HOST)
    assert rc == hs.HSAD_E_INVALID_DATA
    import torch
    rc, _ = hs.hsad_push_lines(det.ctx, torch.from_numpy(x).cuda(), 4, hs.HSAD_DEVICE)
    assert rc == hs.HSAD_E_INVALID_DATA
    det.close()


def test_scores_poll_and_ring_eviction(hs):
    sc, lines = _scene_lines(20, 32, 8, seed=4)
    det = hs.Detector(width=32, bands=8, stats_mode="exclusive", result_lines=8, max_batch_lines=4)
    rc, _ = hs.hsad_push_lines(det.ctx, lines[:8], 8, hs.HSAD_HOST)
    assert rc == hs.HSAD_OK
    rc, _ = hs.hsad_push_lines(det.ctx, lines[8:16], 8, hs.HSAD_HOST)
    assert rc == hs.HSAD_OK
    s = np.empty((4, 32), np.float32)
    assert hs.hsad_scores(det.ctx, 0, 4, s, None, hs.HSAD_HOST, -1) == hs.HSAD_E_INVALID  # evicted
    assert hs.hsad_scores(det.ctx, 12, 4, s, None, hs.HSAD_HOST, -1) == hs.HSAD_OK
    assert hs.hsad_scores(det.ctx, 16, 1, s, None, hs.HSAD_HOST, -1) == hs.HSAD_E_INVALID  # not pushed
    rc, _ = hs.hsad_push_lines(det.ctx, lines[:9], 9, hs.HSAD_HOST)
    assert rc == hs.HSAD_E_INVALID                                                   # above the ring
    det.close()
