"""Binding of libksdf_peaks.so (include/ksdf_peaks.h): the measured throughput of the execution units the
Kernel-SDF kernels are bound by, used as roofline denominators by the benchmark.  Measurement only; the
library of the method (ksdf.py) does not use it."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libksdf_peaks.so")
UNITS = {"fp64_dfma_tflops": 0, "fp32_ffma_tops": 1, "mufu_ex2_tops": 2, "tf32_tcgen05_tflops": 3,
         "fp32x2_ffma_tops": 4}
_lib = None


def load(path: str = LIB_PATH):
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("libksdf_peaks.so is not built (%s)" % path)
        lib = ctypes.CDLL(path)
        lib.ksdf_peaks_measure.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
        lib.ksdf_peaks_measure.restype = ctypes.c_int
        lib.ksdf_peaks_last_error.argtypes = []
        lib.ksdf_peaks_last_error.restype = ctypes.c_char_p
        _lib = lib
    return _lib


def measure(unit: str, stream: int | None = None, repeats: int = 3) -> float:
    """Best of `repeats` probe runs of one unit (see UNITS) on the current device, in the header's units."""
    lib = load()
    best = 0.0
    for _ in range(repeats):
        r = ctypes.c_double(0.0)
        rc = lib.ksdf_peaks_measure(UNITS[unit], stream, ctypes.byref(r))
        if rc != 0:
            raise RuntimeError("ksdf_peaks_measure(%s): %s" % (unit, lib.ksdf_peaks_last_error().decode()))
        best = max(best, r.value)
    return best


def measure_all(stream: int | None = None) -> dict:
    """Every unit's rate; a unit whose probe failed maps to None (its message under "<unit>_error")."""
    out = {}
    for k in UNITS:
        try:
            out[k] = measure(k, stream)
        except RuntimeError as e:
            out[k] = None
            out[k + "_error"] = str(e)
    return out
