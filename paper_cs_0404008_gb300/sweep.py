"""Binding of libgfpsweep: host (CPU) implementations of the dot-product
representations compared in Section 3 of the paper (Figures 5-8), used to
time sweeps over the modulus on the host cores.

Marshalling only; the arithmetic is in ``sweep/gfp_sweep.c`` and the
interface in ``include/gfpsweep.h``.  This is a measurement component: the GPU
library never calls it.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build

# variant ids of include/gfpsweep.h, in order
VARIANTS = ["zpz32", "block32", "overflow32", "hybrid32", "centered_block32",
            "centered_overflow32", "montgomery_block16", "zpz64", "block64", "overflow64",
            "hybrid64", "fp53_block", "montgomery_block32"]
WORD32 = VARIANTS[:7]
WORD64 = VARIANTS[7:]

ERR_DOMAIN = -1
ERR_ARG = -2

_u32p = ctypes.POINTER(ctypes.c_uint32)
_lib = None


def lib():
    """Load libgfpsweep (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        so = ctypes.CDLL(_build.build_sweep())
        so.gfp_sweep_name.restype = ctypes.c_char_p
        so.gfp_sweep_name.argtypes = [ctypes.c_int]
        so.gfp_sweep_supported.restype = ctypes.c_int
        so.gfp_sweep_supported.argtypes = [ctypes.c_int, ctypes.c_uint32]
        so.gfp_sweep_block.restype = ctypes.c_uint64
        so.gfp_sweep_block.argtypes = [ctypes.c_int, ctypes.c_uint32]
        so.gfp_sweep_dot.restype = ctypes.c_int
        so.gfp_sweep_dot.argtypes = [ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, _u32p, _u32p,
                                     _u32p]
        so.gfp_sweep_time.restype = ctypes.c_int
        so.gfp_sweep_time.argtypes = [ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, _u32p, _u32p,
                                      ctypes.c_uint64, ctypes.POINTER(ctypes.c_double), _u32p]
        _lib = so
    return _lib


def _vid(v) -> int:
    return VARIANTS.index(v) if isinstance(v, str) else int(v)


def _vec(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


def name(v) -> str:
    r = lib().gfp_sweep_name(_vid(v))
    return r.decode() if r else None


def supported(v, p: int) -> bool:
    return bool(lib().gfp_sweep_supported(_vid(v), p))


def block(v, p: int) -> int:
    return int(lib().gfp_sweep_block(_vid(v), p))


def dot(v, p: int, x, y) -> int:
    """Canonical residue of sum x_i y_i mod p through variant v."""
    x, y = _vec(x), _vec(y)
    assert x.shape == y.shape and x.ndim == 1
    out = ctypes.c_uint32()
    st = lib().gfp_sweep_dot(_vid(v), p, x.shape[0], x.ctypes.data_as(_u32p),
                             y.ctypes.data_as(_u32p), ctypes.byref(out))
    if st != 0:
        raise ValueError(f"gfp_sweep_dot({name(v)}, p={p}) failed with {st}")
    return int(out.value)


def time(v, p: int, x, y, reps: int):
    """(seconds for `reps` back-to-back dot products, residue)."""
    x, y = _vec(x), _vec(y)
    assert x.shape == y.shape and x.ndim == 1
    sec = ctypes.c_double()
    out = ctypes.c_uint32()
    st = lib().gfp_sweep_time(_vid(v), p, x.shape[0], x.ctypes.data_as(_u32p),
                              y.ctypes.data_as(_u32p), reps, ctypes.byref(sec), ctypes.byref(out))
    if st != 0:
        raise ValueError(f"gfp_sweep_time({name(v)}, p={p}) failed with {st}")
    return float(sec.value), int(out.value)
