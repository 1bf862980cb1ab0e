"""Binding of libgfppeaks: the hardware ceilings (read-only and copy HBM
streams, L2 reads, DFMA, warp-level s8 MMA, graph launch floor) measured by
this project's own kernels, for the rooflines that bench.py reports.

Marshalling only; the kernels are in ``peaks/gfp_peaks.cu`` and the interface
in ``include/gfppeaks.h``.  A measurement component: libgfpdot never calls it.
"""
from __future__ import annotations

import ctypes

from . import build as _build

KINDS = ["read_hbm", "copy_hbm", "read_l2", "dfma", "imma_sync_s8", "launch"]
UNITS = {"read_hbm": "GB/s", "copy_hbm": "GB/s", "read_l2": "GB/s", "dfma": "TFLOP/s",
         "imma_sync_s8": "TOP/s", "launch": "us per launch"}


class gfp_peak_result(ctypes.Structure):
    _fields_ = [("rate", ctypes.c_double), ("rate_median", ctypes.c_double),
                ("ms_best", ctypes.c_double), ("ms_median", ctypes.c_double),
                ("work", ctypes.c_double), ("grid", ctypes.c_int), ("threads", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        so = ctypes.CDLL(_build.build_peaks())
        so.gfp_peak_measure.restype = ctypes.c_int
        so.gfp_peak_measure.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                        ctypes.POINTER(gfp_peak_result)]
        so.gfp_peak_name.restype = ctypes.c_char_p
        so.gfp_peak_name.argtypes = [ctypes.c_int]
        _lib = so
    return _lib


def measure(kind: str, nbytes: int = 0, reps: int = 10) -> dict:
    """Run one probe on the current device; returns its figures as a dict."""
    r = gfp_peak_result()
    st = lib().gfp_peak_measure(KINDS.index(kind), nbytes, reps, ctypes.byref(r))
    if st != 0:
        raise RuntimeError(f"gfp_peak_measure({kind}) failed with status {st}")
    return {"kind": kind, "rate": r.rate, "rate_median": r.rate_median, "unit": UNITS[kind],
            "ms_best": r.ms_best, "ms_median": r.ms_median, "work": r.work, "grid": r.grid,
            "threads": r.threads}
