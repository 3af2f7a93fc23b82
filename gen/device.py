"""Device-resident synthetic push-broom cubes (for workloads too large to draw on the host).

Draws DN with the scene parameters of a host :class:`gen.cubes.PushbroomScene` on the
GPU (gen/csrc/gen_device.cu). Differences from the host recipe, stated here once: shot
noise uses the normal approximation N(s, q s) of q * Poisson(s / q), anomalies are
isolated pixels with probability ``anomaly_fraction``, and the random streams are
Philox4x32-10 keyed by ``seed`` and the pixel index (so values differ from the host
generator's). Nothing here computes a statistic of the data.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "libhsadgen.so")


class _Scene(C.Structure):
    _fields_ = [("W", C.c_int), ("B", C.c_int), ("K", C.c_int),
                ("materials", C.c_void_p), ("illum", C.c_void_p), ("offset", C.c_void_p),
                ("q", C.c_void_p), ("anomaly", C.c_void_p),
                ("a", C.c_float * 8), ("b", C.c_float * 8), ("period", C.c_float * 8),
                ("phase", C.c_float * 8), ("c", C.c_float * 8), ("xfreq", C.c_float * 8),
                ("xphase", C.c_float * 8),
                ("amplitude", C.c_float), ("rho", C.c_float), ("read_noise", C.c_float),
                ("anomaly_fraction", C.c_float)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise ImportError(f"{LIB} missing: run __graft_entry__.build()")
        _lib = C.CDLL(LIB)
        _lib.hsadgen_pushbroom.restype = C.c_int
        _lib.hsadgen_pushbroom.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_uint64, C.c_void_p]
        _lib.hsadgen_scene_size.restype = C.c_int
        assert _lib.hsadgen_scene_size() == C.sizeof(_Scene), "scene struct layout mismatch"
    return _lib


class DeviceScene:
    """Device copy of a PushbroomScene's parameters; ``generate`` fills a cuda tensor."""

    def __init__(self, scene, device="cuda"):
        import torch
        self.scene = scene
        f = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device=device).contiguous()  # noqa: E731
        self._keep = [f(scene.materials), f(scene.illum), f(scene.offset), f(scene.q), f(scene.anomaly_spectra)]
        K = scene.materials.shape[0]
        p = _Scene(W=scene.width, B=scene.bands, K=K)
        p.materials, p.illum, p.offset, p.q, p.anomaly = [t.data_ptr() for t in self._keep]
        for name, arr in (("a", scene.a), ("b", scene.b), ("period", scene.period), ("phase", scene.phase),
                          ("c", scene.c), ("xfreq", scene.xfreq), ("xphase", scene.xphase)):
            getattr(p, name)[:K] = [float(v) for v in arr]
        p.amplitude, p.rho = float(scene.amplitude), float(scene.rho)
        p.read_noise, p.anomaly_fraction = float(scene.read_noise), float(scene.anomaly_fraction)
        self.params = p

    def generate(self, out, t0: int = 0, seed: int = 1, stream: int = 0):
        """Fill ``out`` (cuda tensor of 2-byte elements, [n_lines, W, B]) with lines t0.. ."""
        lib = _load()
        n = out.shape[0]
        assert out.is_cuda and out.is_contiguous() and out.element_size() == 2
        assert tuple(out.shape[1:]) == (self.scene.width, self.scene.bands)
        rc = lib.hsadgen_pushbroom(C.addressof(self.params), out.data_ptr(), int(t0), int(n), int(seed), stream)
        if rc != 0:
            raise RuntimeError(f"device generator failed ({rc})")
        return out
