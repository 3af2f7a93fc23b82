"""C ABI contract checks that need no GPU: symbols, validation, NULL handling."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hs():
    import importlib.util
    spec = importlib.util.spec_from_file_location("hsad_build", os.path.join(ROOT, "paper_2602_13509_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()                      # cross-compiles for sm_103a; no GPU needed
    import paper_2602_13509_gb300 as hs
    return hs


def test_library_exports_every_declared_function(hs):
    names = hs.header_functions()
    assert {"hsad_create", "hsad_push_lines", "hsad_scores", "hsad_destroy", "hsad_last_error"} <= set(names)
    lib = hs.library()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_header_is_plain_c():
    txt = open(os.path.join(ROOT, "include", "hsad.h")).read()
    assert 'extern "C"' in txt
    assert not re.search(r"\b(torch|at::|Tensor|std::)", txt)


def test_config_defaults_and_struct_size(hs):
    cfg = hs.hsad_config_init()
    assert cfg.in_dtype == hs.HSAD_U16 and cfg.precision == hs.HSAD_FP32
    assert cfg.stats_mode == hs.HSAD_EXCLUSIVE and cfg.threshold_mode == hs.HSAD_ABS
    # 80 + the front-end, cadence, forgetting and factor-precision fields (the last fills
    # the 4-byte tail padding of the 8-byte aligned struct)
    assert C.sizeof(hs.hsad_config) == 104
    assert hs.hsad_config.factor_precision.offset == 100
    assert cfg.raw_bands == 0 and cfg.band_first == 0 and cfg.band_bin == 0   # front end off
    assert cfg.forget == 0.0                                                  # forgetting off
    assert cfg.factor_precision == hs.HSAD_FACTOR_FF                          # float-float factor


@pytest.mark.parametrize("field,value,msg", [
    ("width", 0, "width"), ("bands", 0, "bands"), ("bands", 513, "bands"), ("in_dtype", 7, "in_dtype"),
    ("precision", 9, "precision"), ("stats_mode", 5, "stats_mode"), ("cube_lines", -1, "cube_lines"),
    ("threshold_mode", 4, "threshold_mode"), ("threshold", -1.0, "threshold"),
    ("warmup_pixels", -5, "warmup"), ("max_batch_lines", 70000, "max_batch_lines"), ("flags", 64, "flags"),
    ("forget", 1.5, "forget"), ("forget", -0.25, "forget"), ("forget", float("nan"), "forget"),
    ("factor_precision", 2, "factor_precision"), ("factor_precision", -1, "factor_precision"),
    ("flags", 16, "flags"),
])
def test_create_rejects_bad_fields(hs, field, value, msg):
    cfg = hs.make_config(64, 32)
    setattr(cfg, field, value)
    rc, ctx = hs.hsad_create(cfg)
    assert rc == hs.HSAD_E_INVALID and ctx is None
    assert msg.split("_")[0] in hs.hsad_last_error(None)


def test_create_rejects_inconsistent_modes(hs):
    assert hs.hsad_create(hs.make_config(8, 4, stats_mode="cube"))[0] == hs.HSAD_E_INVALID       # no cube_lines
    assert hs.hsad_create(hs.make_config(8, 4, threshold_mode="rel"))[0] == hs.HSAD_E_INVALID     # REL needs cube
    assert hs.hsad_create(hs.make_config(8, 4, flags=hs.HSAD_NORMALIZE_SCORES))[0] == hs.HSAD_E_INVALID
    assert hs.hsad_create(hs.make_config(8, 4, gain=[1, 0, 1, 1]))[0] == hs.HSAD_E_INVALID        # zero gain
    assert hs.hsad_create(hs.make_config(8, 4, gain=[1, float("nan"), 1, 1]))[0] == hs.HSAD_E_INVALID
    # forgetting needs streamed statistics and does not combine with a cadence
    assert hs.hsad_create(hs.make_config(8, 4, stats_mode="cube", cube_lines=4, forget=0.9))[0] == hs.HSAD_E_INVALID
    assert hs.hsad_create(hs.make_config(8, 4, factor_every=2, forget=0.9))[0] == hs.HSAD_E_INVALID
    assert "forget" in hs.hsad_last_error(None)


def test_null_handling(hs):
    lib = hs.library()
    assert hs.hsad_destroy(None) == hs.HSAD_OK
    assert hs.hsad_push_lines(None, None, 1, hs.HSAD_HOST)[0] == hs.HSAD_E_INVALID
    assert hs.hsad_scores(None, 0, 1, None, None, hs.HSAD_HOST, 0) == hs.HSAD_E_INVALID
    assert hs.hsad_flush(None) == hs.HSAD_E_INVALID
    assert hs.hsad_reset(None) == hs.HSAD_E_INVALID
    assert hs.hsad_synchronize(None, 0) == hs.HSAD_E_INVALID
    assert lib.hsad_create(None, None) == hs.HSAD_E_INVALID
    assert lib.hsad_config_init(None) == hs.HSAD_E_INVALID
    assert isinstance(hs.hsad_last_error(None), str)
    assert hs.hsad_stream(None) == 0 and hs.hsad_kernel_launches(None) == 0
    assert hs.hsad_whitening_form(None) == hs.HSAD_E_INVALID


def test_status_strings(hs):
    for code in range(0, -9, -1):
        assert hs.hsad_status_string(code).startswith("HSAD_")
    assert hs.hsad_status_string(42) == "unknown status"


def test_valid_config_without_gpu_reports_cuda_error(hs):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rc, ctx = hs.hsad_create(hs.make_config(640, 270))
    assert rc == hs.HSAD_E_CUDA and ctx is None


def test_budget_calls_are_host_only(hs):
    assert hs.hsad_set_device_budget(0, -1) == hs.HSAD_E_INVALID
    assert hs.hsad_set_device_budget(0, 0) == hs.HSAD_OK
    assert hs.hsad_device_budget_used(0) == 0


def test_create_rejects_bad_front_end(hs):
    def rc(**kw):
        r, ctx = hs.hsad_create(hs.make_config(16, 8, **kw))
        return r, hs.hsad_last_error(None)
    assert rc(raw_bands=-1)[0] == hs.HSAD_E_INVALID
    r, why = rc(raw_bands=40, band_bin=5)
    assert r == hs.HSAD_E_INVALID and "band_bin" in why
    r, why = rc(raw_bands=40, band_first=10, band_bin=4)          # 10 + 4 * 8 > 40
    assert r == hs.HSAD_E_INVALID and "raw_bands" in why
    r, why = rc(raw_bands=40, band_bin=4, in_dtype="f32")
    assert r == hs.HSAD_E_INVALID and "U16" in why


def test_create_rejects_bad_cadence(hs):
    for kw in (dict(factor_every=-1), dict(factor_every=65), dict(factor_every=2, stats_mode="inclusive")):
        r, ctx = hs.hsad_create(hs.make_config(16, 8, **kw))
        assert r == hs.HSAD_E_INVALID and "factor_every" in hs.hsad_last_error(None)
