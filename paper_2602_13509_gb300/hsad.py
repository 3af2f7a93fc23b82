"""Thin ctypes binding of the hsad C ABI (include/hsad.h).

Every function here has the same name as its C entry point and only marshals
arguments: numpy arrays and torch tensors become raw pointers, status codes
come back unchanged. All computation happens in the CUDA library
``libhsad.so``; if that library is missing, importing this module fails.
"""
from __future__ import annotations

import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhsad.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "hsad.h")

# status codes
HSAD_OK, HSAD_E_INVALID, HSAD_E_NOMEM, HSAD_E_NOT_READY = 0, -1, -2, -3
HSAD_E_NOT_PD, HSAD_E_TIMEOUT, HSAD_E_CUDA, HSAD_E_BUSY, HSAD_E_INVALID_DATA = -4, -5, -6, -7, -8
# enums
HSAD_U16, HSAD_F32 = 0, 1
HSAD_FP32, HSAD_BF16, HSAD_FP16 = 0, 1, 2
HSAD_FORM_INVERSE, HSAD_FORM_TRIANGULAR_SOLVE = 0, 1
HSAD_EXCLUSIVE, HSAD_INCLUSIVE, HSAD_CUBE = 0, 1, 2
HSAD_ABS, HSAD_REL = 0, 1
HSAD_HOST, HSAD_DEVICE = 0, 1
HSAD_CREATE_WAIT, HSAD_NORMALIZE_SCORES, HSAD_CUDA_GRAPHS, HSAD_FORCE_INVERSE = 1, 2, 4, 8
HSAD_FACTOR_FF, HSAD_FACTOR_FP64 = 0, 1
# per-line status
LS_OK, LS_NOT_READY, LS_NOT_PD, LS_INVALID_DATA = 0, 1, 2, 3


class hsad_config(C.Structure):
    _fields_ = [
        ("width", C.c_int32), ("bands", C.c_int32), ("in_dtype", C.c_int32),
        ("precision", C.c_int32), ("stats_mode", C.c_int32), ("cube_lines", C.c_int32),
        ("gain", C.POINTER(C.c_float)), ("offset", C.POINTER(C.c_float)),
        ("threshold_mode", C.c_int32), ("threshold", C.c_float),
        ("warmup_pixels", C.c_int64), ("device_budget_bytes", C.c_int64),
        ("flags", C.c_int32), ("device", C.c_int32),
        ("max_batch_lines", C.c_int32), ("result_lines", C.c_int32),
        ("raw_bands", C.c_int32), ("band_first", C.c_int32), ("band_bin", C.c_int32),
        ("factor_every", C.c_int32),
        ("forget", C.c_float),
        ("factor_precision", C.c_int32),
    ]


class HsadError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{hsad_status_string(code)}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"hsad CUDA library not built ({LIB_PATH} missing); run "
            "`python -c 'import __graft_entry__ as g; g.build()'` first. There is no fallback.")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    sig = {
        "hsad_config_init": (C.c_int, [C.POINTER(hsad_config)]),
        "hsad_create": (C.c_int, [C.POINTER(hsad_config), C.POINTER(P)]),
        "hsad_push_lines": (C.c_int, [P, P, C.c_int64, C.c_int32, C.POINTER(C.c_uint64)]),
        "hsad_push_lines_gain": (C.c_int, [P, P, P, C.c_int64, C.c_int32, C.POINTER(C.c_uint64)]),
        "hsad_flush": (C.c_int, [P]),
        "hsad_scores": (C.c_int, [P, C.c_uint64, C.c_int64, P, P, C.c_int32, C.c_int32]),
        "hsad_scores_tx": (C.c_int, [P, C.c_uint64, C.c_int64, P, C.POINTER(C.c_float), C.c_int32, C.c_int32]),
        "hsad_encode_scores": (C.c_int, [P, C.c_int64, P, C.POINTER(C.c_float), C.c_int32, P]),
        "hsad_frontend": (C.c_int, [P, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P, C.c_int32, P]),
        "hsad_line_status": (C.c_int, [P, C.c_uint64, C.c_int64, P, C.c_int32]),
        "hsad_synchronize": (C.c_int, [P, C.c_int32]),
        "hsad_reset": (C.c_int, [P]),
        "hsad_get_stats": (C.c_int, [P, C.POINTER(C.c_int64), P, P, P]),
        "hsad_stream": (P, [P]),
        "hsad_kernel_launches": (C.c_int64, [P]),
        "hsad_device_bytes": (C.c_int64, [P]),
        "hsad_whitening_form": (C.c_int, [P]),
        "hsad_whitening_tensor_cores": (C.c_int, [P]),
        "hsad_set_device_budget": (C.c_int, [C.c_int, C.c_int64]),
        "hsad_device_budget_used": (C.c_int64, [C.c_int]),
        "hsad_profile_enable": (C.c_int, [P, C.c_int32]),
        "hsad_profile_read": (C.c_int, [P, C.c_int32, C.c_char_p, C.c_int32, C.POINTER(C.c_int64),
                                        C.POINTER(C.c_double)]),
        "hsad_profile_reset": (C.c_int, [P]),
        "hsad_global_rx_noalloc": (C.c_int, [P, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                             C.POINTER(C.c_float), C.c_int32, C.c_float, C.c_int32, P, P, P,
                                             C.c_int32]),
        "hsad_krx": (C.c_int, [P, C.c_int64, C.c_int32, C.c_int32, P, C.c_int32, C.c_float, C.c_float,
                               C.POINTER(C.c_float), C.c_int32, C.c_float, C.c_int32, P, P, P, C.c_int32]),
        "hsad_engine_create": (C.c_int, [C.c_int32, C.c_int64, C.POINTER(P)]),
        "hsad_engine_open": (C.c_int, [P, C.POINTER(hsad_config), C.POINTER(C.c_int32)]),
        "hsad_engine_submit": (C.c_int, [P, C.c_int32, P, C.c_int64, C.POINTER(C.c_uint64)]),
        "hsad_engine_results": (C.c_int, [P, C.c_int32, C.c_uint64, C.c_int64, P, P, C.c_int32]),
        "hsad_engine_close": (C.c_int, [P, C.c_int32]),
        "hsad_engine_counters": (C.c_int, [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
        "hsad_engine_destroy": (C.c_int, [P]),
        "hsad_selftest_bounded_wait": (C.c_int, [C.c_int32, C.c_int64, C.POINTER(C.c_int32)]),
        "hsad_set_stats": (C.c_int, [P, C.c_int64, P, P, P]),
        "hsad_autotune_factor": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_float),
                                           C.POINTER(C.c_int32)]),
        "hsad_destroy": (C.c_int, [P]),
        "hsad_last_error": (C.c_char_p, [P]),
        "hsad_status_string": (C.c_char_p, [C.c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    return lib


_lib = _load()


def header_functions() -> list[str]:
    """Names of every function declared in include/hsad.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hsad_[a-z_0-9]+)\s*\(", txt)))


def library():
    return _lib


def _ptr(a) -> int | None:
    """Raw address of a numpy array or torch tensor (None stays None)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if hasattr(a, "ctypes"):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if isinstance(a, int):
        return a
    raise TypeError(f"cannot take the address of {type(a)}")


# ---------------------------------------------------------------- C entry points
def hsad_status_string(code: int) -> str:
    return _lib.hsad_status_string(int(code)).decode()


def hsad_last_error(ctx=None) -> str:
    return (_lib.hsad_last_error(ctx) or b"").decode()


def hsad_config_init(cfg: hsad_config | None = None) -> hsad_config:
    cfg = cfg or hsad_config()
    _lib.hsad_config_init(C.byref(cfg))
    return cfg


def hsad_create(cfg: hsad_config):
    """Returns ``(status, ctx)``; ctx is an opaque handle (int) or None."""
    out = C.c_void_p()
    rc = _lib.hsad_create(C.byref(cfg), C.byref(out))
    return rc, (out.value if rc == HSAD_OK else None)


def hsad_push_lines(ctx, lines, n_lines: int, mem: int):
    """Returns ``(status, first_line_id)``."""
    first = C.c_uint64(0)
    rc = _lib.hsad_push_lines(ctx, _ptr(lines), int(n_lines), int(mem), C.byref(first))
    return rc, first.value


def hsad_push_lines_gain(ctx, lines, line_gain, n_lines: int, mem: int):
    """Push lines recorded at per-line gains ``line_gain`` (host float32, one per line).
    Returns ``(status, first_line_id)``."""
    first = C.c_uint64(0)
    rc = _lib.hsad_push_lines_gain(ctx, _ptr(lines), _ptr(line_gain), int(n_lines), int(mem), C.byref(first))
    return rc, first.value


def hsad_flush(ctx) -> int:
    return _lib.hsad_flush(ctx)


def hsad_scores(ctx, first_line_id: int, n_lines: int, scores, mask, mem: int, timeout_ms: int) -> int:
    return _lib.hsad_scores(ctx, int(first_line_id), int(n_lines), _ptr(scores), _ptr(mask), int(mem),
                            int(timeout_ms))


def hsad_scores_tx(ctx, first_line_id: int, n_lines: int, codes, mem: int, timeout_ms: int):
    """Transmit codes (binary16 of sqrt(delta / delta_max)) of a block of lines into ``codes``
    (uint16, n_lines x width). Returns ``(status, delta_max)``."""
    mx = C.c_float(0.0)
    rc = _lib.hsad_scores_tx(ctx, int(first_line_id), int(n_lines), _ptr(codes), C.byref(mx), int(mem),
                             int(timeout_ms))
    return rc, mx.value


def hsad_frontend(raw, n_pixels: int, raw_bands: int, band_first: int, band_bin: int, bands: int, out,
                  device: int = 0, stream=None) -> int:
    return _lib.hsad_frontend(_ptr(raw), int(n_pixels), int(raw_bands), int(band_first), int(band_bin), int(bands),
                              _ptr(out), int(device), _ptr(stream))


def hsad_encode_scores(scores, n: int, codes, device: int = 0, stream=None):
    """Transmit codes of n device scores into n device codes. Returns ``(status, delta_max)``."""
    mx = C.c_float(0.0)
    rc = _lib.hsad_encode_scores(_ptr(scores), int(n), _ptr(codes), C.byref(mx), int(device), _ptr(stream))
    return rc, mx.value


def hsad_line_status(ctx, first_line_id: int, n_lines: int, status, timeout_ms: int) -> int:
    return _lib.hsad_line_status(ctx, int(first_line_id), int(n_lines), _ptr(status), int(timeout_ms))


def hsad_synchronize(ctx, timeout_ms: int = -1) -> int:
    return _lib.hsad_synchronize(ctx, int(timeout_ms))


def hsad_reset(ctx) -> int:
    return _lib.hsad_reset(ctx)


def hsad_get_stats(ctx, bands: int):
    """Returns ``(status, n_pixels, shift [B], s1 [B], s2 [B, B])`` as numpy arrays."""
    import numpy as np
    n = C.c_int64(0)
    c = np.zeros(bands, np.float64)
    s1 = np.zeros(bands, np.float64)
    s2 = np.zeros((bands, bands), np.float64)
    rc = _lib.hsad_get_stats(ctx, C.byref(n), c.ctypes.data, s1.ctypes.data, s2.ctypes.data)
    return rc, n.value, c, s1, s2


def hsad_stream(ctx) -> int:
    return _lib.hsad_stream(ctx) or 0


def hsad_kernel_launches(ctx) -> int:
    return int(_lib.hsad_kernel_launches(ctx))


def hsad_device_bytes(ctx) -> int:
    return int(_lib.hsad_device_bytes(ctx))


def hsad_whitening_form(ctx) -> int:
    return int(_lib.hsad_whitening_form(ctx))


def hsad_whitening_tensor_cores(ctx) -> int:
    return int(_lib.hsad_whitening_tensor_cores(ctx))


def hsad_set_device_budget(device: int, nbytes: int) -> int:
    return _lib.hsad_set_device_budget(int(device), int(nbytes))


def hsad_device_budget_used(device: int) -> int:
    return int(_lib.hsad_device_budget_used(int(device)))


def hsad_profile_enable(ctx, enable: bool) -> int:
    return _lib.hsad_profile_enable(ctx, 1 if enable else 0)


def hsad_profile_read(ctx, index: int):
    """Returns ``(status, name, launches, total_ms)``."""
    buf = C.create_string_buffer(64)
    n, ms = C.c_int64(0), C.c_double(0.0)
    rc = _lib.hsad_profile_read(ctx, int(index), buf, 64, C.byref(n), C.byref(ms))
    return rc, buf.value.decode(), n.value, ms.value


def hsad_profile_reset(ctx) -> int:
    return _lib.hsad_profile_reset(ctx)


def hsad_krx(cube, n_pixels, bands, in_dtype, subsample, kernel_width, ridge, gain, threshold_mode, threshold,
             flags, scores, mask, stream=None, device=0) -> int:
    """Subsampled kernel RX of one device cube (see include/hsad.h); ``subsample``: host
    int64 pixel indices."""
    import numpy as np
    idx = np.ascontiguousarray(np.asarray(subsample, dtype=np.int64).reshape(-1))
    g = None
    if gain is not None:
        keep = np.ascontiguousarray(np.asarray(gain, dtype=np.float32))
        g = keep.ctypes.data_as(C.POINTER(C.c_float))
    return _lib.hsad_krx(_ptr(cube), int(n_pixels), int(bands), int(in_dtype), idx.ctypes.data, int(idx.size),
                         float(kernel_width), float(ridge), g, int(threshold_mode), float(threshold), int(flags),
                         _ptr(scores), _ptr(mask), stream, int(device))


def hsad_global_rx_noalloc(cube, n_lines, width, bands, in_dtype, precision, gain, threshold_mode,
                           threshold, flags, scores, mask, stream=None, device=0) -> int:
    """Allocation-free global RX of one device cube (see include/hsad.h)."""
    g = None
    if gain is not None:
        import numpy as np
        keep = np.ascontiguousarray(np.asarray(gain, dtype=np.float32))
        g = keep.ctypes.data_as(C.POINTER(C.c_float))
    return _lib.hsad_global_rx_noalloc(_ptr(cube), int(n_lines), int(width), int(bands), int(in_dtype),
                                       int(precision), g, int(threshold_mode), float(threshold), int(flags),
                                       _ptr(scores), _ptr(mask), stream, int(device))


def hsad_engine_create(device: int = 0, budget_bytes: int = 0):
    """Returns ``(status, engine)``."""
    out = C.c_void_p()
    rc = _lib.hsad_engine_create(int(device), int(budget_bytes), C.byref(out))
    return rc, (out.value if rc == HSAD_OK else None)


def hsad_engine_open(engine, cfg: hsad_config):
    """Returns ``(status, stream_id)``."""
    sid = C.c_int32(-1)
    rc = _lib.hsad_engine_open(engine, C.byref(cfg), C.byref(sid))
    return rc, sid.value


def hsad_engine_submit(engine, stream_id: int, lines, n_lines: int):
    """Returns ``(status, first_line_id)``."""
    first = C.c_uint64(0)
    rc = _lib.hsad_engine_submit(engine, int(stream_id), _ptr(lines), int(n_lines), C.byref(first))
    return rc, first.value


def hsad_engine_results(engine, stream_id: int, first: int, n_lines: int, scores, mask, timeout_ms: int = -1):
    return _lib.hsad_engine_results(engine, int(stream_id), int(first), int(n_lines), _ptr(scores), _ptr(mask),
                                    int(timeout_ms))


def hsad_engine_close(engine, stream_id: int) -> int:
    return _lib.hsad_engine_close(engine, int(stream_id))


def hsad_engine_counters(engine):
    """Returns ``(last_error, lines, pushes, max_batch)``."""
    a, b, c = C.c_int64(0), C.c_int64(0), C.c_int64(0)
    rc = _lib.hsad_engine_counters(engine, C.byref(a), C.byref(b), C.byref(c))
    return rc, a.value, b.value, c.value


def hsad_engine_destroy(engine) -> int:
    return _lib.hsad_engine_destroy(engine)


def hsad_set_stats(ctx, n_pixels: int, shift, s1, s2) -> int:
    """Import statistics exported by hsad_get_stats (float64 numpy arrays)."""
    import numpy as np
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (shift, s1, s2)]
    return _lib.hsad_set_stats(ctx, int(n_pixels), *(a.ctypes.data for a in arrs))


def hsad_autotune_factor(device: int, bands: int, precision: str, max_lines: int):
    """Returns ``(status, rows)``, rows = [(bucket, ctas_per_line, threads, ms), ...]."""
    cap = 16
    buf = (C.c_float * (4 * cap))()
    n = C.c_int32(cap)
    rc = _lib.hsad_autotune_factor(int(device), int(bands), _NAMES[precision], int(max_lines), buf, C.byref(n))
    rows = [tuple(buf[4 * i:4 * i + 4]) for i in range(min(n.value, cap))] if rc == HSAD_OK else []
    return rc, rows


def hsad_selftest_bounded_wait(device: int = 0, limit_cycles: int = 2_000_000):
    """Returns ``(status, timed_out)``."""
    flag = C.c_int32(-1)
    rc = _lib.hsad_selftest_bounded_wait(int(device), int(limit_cycles), C.byref(flag))
    return rc, flag.value


def hsad_destroy(ctx) -> int:
    return _lib.hsad_destroy(ctx)


# ---------------------------------------------------------------- convenience wrapper
_NAMES = {
    "u16": HSAD_U16, "f32": HSAD_F32,
    "fp32": HSAD_FP32, "bf16": HSAD_BF16, "fp16": HSAD_FP16,
    "exclusive": HSAD_EXCLUSIVE, "inclusive": HSAD_INCLUSIVE, "cube": HSAD_CUBE,
    "abs": HSAD_ABS, "rel": HSAD_REL,
}


def make_config(width, bands, in_dtype="u16", precision="fp32", stats_mode="exclusive", cube_lines=0,
                gain=None, offset=None, threshold_mode="abs", threshold=0.0, warmup_pixels=0,
                device_budget_bytes=0, flags=0, device=0, max_batch_lines=0, result_lines=0,
                raw_bands=0, band_first=0, band_bin=1, factor_every=0, forget=0.0, factor_precision="ff"):
    """Build an hsad_config; ``gain``/``offset`` arrays are kept alive on the struct."""
    import numpy as np
    cfg = hsad_config_init()
    cfg.width, cfg.bands = int(width), int(bands)
    cfg.in_dtype = _NAMES.get(in_dtype, in_dtype)
    cfg.precision = _NAMES.get(precision, precision)
    cfg.stats_mode = _NAMES.get(stats_mode, stats_mode)
    cfg.cube_lines = int(cube_lines)
    cfg.threshold_mode = _NAMES.get(threshold_mode, threshold_mode)
    cfg.threshold = float(threshold)
    cfg.warmup_pixels, cfg.device_budget_bytes = int(warmup_pixels), int(device_budget_bytes)
    cfg.flags, cfg.device = int(flags), int(device)
    cfg.max_batch_lines, cfg.result_lines = int(max_batch_lines), int(result_lines)
    cfg.raw_bands, cfg.band_first, cfg.band_bin = int(raw_bands), int(band_first), int(band_bin)
    cfg.factor_every = int(factor_every)
    cfg.forget = float(forget)
    cfg.factor_precision = {"ff": HSAD_FACTOR_FF, "fp64": HSAD_FACTOR_FP64}.get(factor_precision, factor_precision)
    keep = []
    for name, arr in (("gain", gain), ("offset", offset)):
        if arr is not None:
            a = np.ascontiguousarray(np.asarray(arr, dtype=np.float32))
            keep.append(a)
            setattr(cfg, name, a.ctypes.data_as(C.POINTER(C.c_float)))
    cfg._keep = keep
    return cfg


class Detector:
    """Owns one hsad context; raises HsadError on hard failures."""

    def __init__(self, **kw):
        self.cfg = make_config(**kw)
        rc, self.ctx = hsad_create(self.cfg)
        if rc != HSAD_OK:
            raise HsadError(rc, hsad_last_error(None))
        self.width, self.bands = self.cfg.width, self.cfg.bands

    def push(self, lines, mem=None, gains=None) -> int:
        """Push lines ([n, W, B] numpy array or contiguous tensor); returns the first line id.
        ``gains``: optional per-line gains (n floats; ``hsad_push_lines_gain``)."""
        if mem is None:
            mem = HSAD_DEVICE if (hasattr(lines, "is_cuda") and lines.is_cuda) else HSAD_HOST
        if gains is None:
            rc, first = hsad_push_lines(self.ctx, lines, lines.shape[0], mem)
        else:
            import numpy as np
            g = np.ascontiguousarray(np.asarray(gains, dtype=np.float32).reshape(-1))
            if g.shape[0] != lines.shape[0]:
                raise ValueError("one gain per line")
            rc, first = hsad_push_lines_gain(self.ctx, lines, g, lines.shape[0], mem)
        if rc != HSAD_OK:
            raise HsadError(rc, hsad_last_error(self.ctx))
        return first

    def flush(self):
        rc = hsad_flush(self.ctx)
        if rc != HSAD_OK:
            raise HsadError(rc, hsad_last_error(self.ctx))

    def scores(self, first, n, timeout_ms=-1):
        """Host copies: ``(status, scores float32 [n, W], mask uint8 [n, W], line_status int32 [n])``."""
        import numpy as np
        s = np.empty((n, self.width), dtype=np.float32)
        m = np.empty((n, self.width), dtype=np.uint8)
        rc = hsad_scores(self.ctx, first, n, s, m, HSAD_HOST, timeout_ms)
        if rc in (HSAD_E_INVALID, HSAD_E_CUDA, HSAD_E_TIMEOUT):
            raise HsadError(rc, hsad_last_error(self.ctx))
        st = np.empty(n, dtype=np.int32)
        rc2 = hsad_line_status(self.ctx, first, n, st, 0)
        if rc2 not in (HSAD_OK,):
            raise HsadError(rc2, hsad_last_error(self.ctx))
        return rc, s, m, st

    def scores_tx(self, first, n, timeout_ms=-1):
        """Transmit codes (Sec. 3.4): ``(status, codes uint16 [n, W], delta_max)``."""
        import numpy as np
        codes = np.empty((n, self.width), dtype=np.uint16)
        rc, mx = hsad_scores_tx(self.ctx, first, n, codes, HSAD_HOST, timeout_ms)
        if rc in (HSAD_E_INVALID, HSAD_E_CUDA, HSAD_E_TIMEOUT):
            raise HsadError(rc, hsad_last_error(self.ctx))
        return rc, codes, mx

    def scores_device(self, first, n, scores, mask, timeout_ms=-1) -> int:
        return hsad_scores(self.ctx, first, n, scores, mask, HSAD_DEVICE, timeout_ms)

    def reset(self):
        rc = hsad_reset(self.ctx)
        if rc != HSAD_OK:
            raise HsadError(rc, hsad_last_error(self.ctx))

    def synchronize(self, timeout_ms=-1):
        rc = hsad_synchronize(self.ctx, timeout_ms)
        if rc != HSAD_OK:
            raise HsadError(rc, hsad_last_error(self.ctx))

    @property
    def stream(self) -> int:
        return hsad_stream(self.ctx)

    def profile(self, enable=True):
        hsad_profile_enable(self.ctx, enable)

    def profile_totals(self) -> dict:
        """{kernel class: (launches, total_ms)} since the last reset."""
        out, i = {}, 0
        while True:
            rc, name, n, ms = hsad_profile_read(self.ctx, i)
            if rc != HSAD_OK:
                break
            out[name] = (n, ms)
            i += 1
        return out

    def profile_reset(self):
        hsad_profile_reset(self.ctx)

    @property
    def kernel_launches(self) -> int:
        return hsad_kernel_launches(self.ctx)

    @property
    def device_bytes(self) -> int:
        return hsad_device_bytes(self.ctx)

    @property
    def whitening_form(self) -> int:
        return hsad_whitening_form(self.ctx)

    @property
    def whitening_tensor_cores(self) -> bool:
        return hsad_whitening_tensor_cores(self.ctx) == 1

    def close(self):
        if self.ctx is not None:
            hsad_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
