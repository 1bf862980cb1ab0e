"""Python binding of libgfpdot (ctypes): argument marshalling only.

Every function keeps the name of the C entry point it calls (declared in
``include/gfpdot.h``).  Device operands are torch CUDA tensors of dtype
uint32 (or int32 holding the same bits); the current torch stream is used
unless ``stream`` is given.  A non-OK status raises :class:`GfpError`.  There
is no fallback: if the shared library is missing, importing the functions
raises, and every computation runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

GFP_OK = 0
GFP_PENDING = 1
GFP_ERR_INVALID = -1
GFP_ERR_RANGE = -2
GFP_ERR_UNSUPPORTED = -3
GFP_ERR_NOMEM = -4
GFP_ERR_CUDA = -5
GFP_ERR_AGAIN = -6
GFP_ERR_TIMEOUT = -7
GFP_ERR_UNKNOWN_TICKET = -8
GFP_ERR_CANCELLED = -9

GFP_REPR_AUTO = 0
GFP_REPR_PERTERM = 1
GFP_REPR_U64_BLOCK = 2
GFP_REPR_U64_CARRY = 3
GFP_REPR_FP64 = 4
GFP_REPR_F16TC = 5
GFP_REPR_CENTERED = 6
GFP_REPR_MONTGOMERY = 7
REPR_NAMES = {0: "auto", 1: "perterm", 2: "u64_block", 3: "u64_carry", 4: "fp64", 5: "f16tc",
              6: "centered", 7: "montgomery"}

_vp = ctypes.c_void_p
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64
_int = ctypes.c_int


class GfpError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = f"{where}: {gfp_status_string(status)} ({status})"
        if status == GFP_ERR_CUDA:
            msg += f": {load().gfp_last_cuda_error().decode()}"
        super().__init__(msg)


class gfp_params(ctypes.Structure):
    _fields_ = [("p", _u32), ("corr", _u32), ("k_u64", _u64), ("k_fp64", _u64),
                ("barrett_mu", _u64), ("inv_p", ctypes.c_double), ("fp64_ok", _int),
                ("k_centered", _u64), ("k_montgomery", _u64)]


class gfp_dot_desc(ctypes.Structure):
    _fields_ = [("p", _u32), ("repr", _u32), ("n", _u64), ("x", _vp), ("y", _vp)]


class gfp_server_cfg(ctypes.Structure):
    _fields_ = [("device", _int), ("mem_budget", _u64), ("max_inflight", _u32),
                ("n_streams", _u32), ("queue_capacity", _u32), ("batch_window_us", _u32),
                ("simulate", _u32), ("fail_every", _u32), ("block_sm_percent", _u32)]


class gfp_job(ctypes.Structure):
    _fields_ = [("kind", _u32), ("p", _u32), ("n", _u64), ("nb", _u64), ("matrix", _u64),
                ("x", _vp), ("y", _vp), ("v", _vp), ("seed", _u64)]


class gfp_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("kind", _u32), ("value", _u32), ("batch", _u32),
                ("out_elems", _u64), ("t_submit_ns", _u64), ("t_admit_ns", _u64),
                ("t_start_ns", _u64), ("t_done_ns", _u64)]


class gfp_server_stats(ctypes.Structure):
    _fields_ = [("submitted", _u64), ("admitted", _u64), ("completed", _u64), ("failed", _u64),
                ("cancelled", _u64), ("admission_stalls", _u64), ("dot_launches", _u64),
                ("mem_in_use", _u64), ("mem_peak", _u64), ("mem_budget", _u64),
                ("kernel_launches", _u64)]


GFP_JOB_DOT = 0
GFP_JOB_MATVEC = 1
GFP_JOB_BLOCK = 2


_SIGS = {
    "gfp_status_string": (ctypes.c_char_p, [_int]),
    "gfp_last_cuda_error": (ctypes.c_char_p, []),
    "gfp_delay_bound": (_u64, [_u32, _int, _int]),
    "gfp_get_params": (_int, [_u32, ctypes.POINTER(gfp_params)]),
    "gfp_reduce_u64": (_u32, [_u64, _u32]),
    "gfp_reduce_f64": (ctypes.c_double, [ctypes.c_double, _u32]),
    "gfp_choose_repr": (_int, [_vp, _u32, _u64]),
    "gfp_context_create": (_int, [_int, ctypes.POINTER(_vp)]),
    "gfp_context_destroy": (_int, [_vp]),
    "gfp_set_repr": (_int, [_vp, _int]),
    "gfp_set_validate": (_int, [_vp, _int]),
    "gfp_launch_count": (_u64, [_vp]),
    "gfp_dot": (_int, [_vp, _u32, _u64, _vp, _vp, _vp, _vp]),
    "gfp_dot_batched": (_int, [_vp, ctypes.POINTER(gfp_dot_desc), _u64, _vp, _vp]),
    "gfp_batch_plan_create": (_int, [_vp, ctypes.POINTER(gfp_dot_desc), _u64, ctypes.POINTER(_vp)]),
    "gfp_batch_plan_exec": (_int, [_vp, _vp, _vp]),
    "gfp_batch_plan_info": (_int, [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64)]),
    "gfp_batch_plan_destroy": (_int, [_vp]),
    "gfp_dot_batched_noalloc": (_int, [ctypes.POINTER(gfp_dot_desc), _u64, _vp, _vp]),
    "gfp_dot_batched_host": (_int, [_vp, _u64, _vp, _vp, _vp, _vp, _vp, _u64, _vp, _vp]),
    "gfp_matvec": (_int, [_vp, _u32, _u64, _u64, _vp, _u64, _vp, _vp, _vp]),
    "gfp_matvec_iterate": (_int, [_vp, _u32, _u64, _vp, _u64, _vp, _vp, _u32, _vp]),
    "gfp_matvec_sequence": (_int, [_vp, _u32, _u64, _vp, _u64, _vp, _vp, _u32, _vp, _vp, _vp]),
    "gfp_matmul_block": (_int, [_vp, _u32, _u64, _u64, _u64, _vp, _u64, _vp, _u64, _vp, _u64, _vp]),
    "gfp_block_prepare": (_int, [_vp, _u32, _u64, _u64, _vp, _u64, ctypes.POINTER(_vp)]),
    "gfp_matmul_block_prepared": (_int, [_vp, _vp, _u64, _vp, _u64, _vp, _u64, _vp]),
    "gfp_block_prep_info": (_int, [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u32)]),
    "gfp_block_prep_destroy": (_int, [_vp]),
    "gfp_matmul_block_csr": (_int, [_vp, _u32, _u64, _u64, _u64, _vp, _vp, _vp, _vp, _u64, _vp, _u64,
                                    _vp]),
    "gfp_context_check": (_int, [_vp]),
    "gfp_wait_selftest": (_int, [_u64, _vp]),
    "gfp_tune": (_int, [_vp, _vp, _u32, _u32, _u32, ctypes.c_char_p]),
    "gfp_plan_load": (_int, [_vp, ctypes.c_char_p]),
    "gfp_plan_save": (_int, [_vp, ctypes.c_char_p]),
    "gfp_plan_size": (_u64, [_vp]),
    "gfp_fill_uniform": (_int, [_u32, _u64, _u64, _u64, _u64, _vp, _vp]),
    "gfp_gfq_find_primitive": (_int, [_u32, _u32, _vp]),
    "gfp_gfq_create": (_int, [_int, _u32, _u32, _vp, ctypes.POINTER(_vp)]),
    "gfp_gfq_destroy": (_int, [_vp]),
    "gfp_gfq_info": (_int, [_vp, ctypes.POINTER(_u32), ctypes.POINTER(_u32), ctypes.POINTER(_u32)]),
    "gfp_gfq_to_log": (_int, [_vp, _u64, _vp, _vp, _vp]),
    "gfp_gfq_from_log": (_int, [_vp, _u64, _vp, _vp, _vp]),
    "gfp_gfq_dot": (_int, [_vp, _u64, _vp, _vp, _vp, _vp]),
    "gfp_gfq_check": (_int, [_vp]),
    "gfp_server_create": (_int, [ctypes.POINTER(gfp_server_cfg), ctypes.POINTER(_vp)]),
    "gfp_server_destroy": (_int, [_vp]),
    "gfp_register_matrix": (_int, [_vp, _u32, _u64, _u64, _vp, _u64, ctypes.POINTER(_u64)]),
    "gfp_submit": (_int, [_vp, ctypes.POINTER(gfp_job), ctypes.POINTER(_u64)]),
    "gfp_prepare_matrix": (_int, [_vp, _u64]),
    "gfp_poll": (_int, [_vp, _u64, ctypes.POINTER(gfp_result)]),
    "gfp_wait": (_int, [_vp, _u64, _u64, ctypes.POINTER(gfp_result)]),
    "gfp_result_copy": (_int, [_vp, _u64, _vp, _u64]),
    "gfp_release": (_int, [_vp, _u64]),
    "gfp_server_get_stats": (_int, [_vp, ctypes.POINTER(gfp_server_stats)]),
}

_lib = None


def load(auto_build: bool = True):
    """Load the in-tree libgfpdot.so (building it first when stale).  The
    environment variable GFPDOT_SANITIZED=1 selects the host-sanitized build
    instead (AddressSanitizer and UndefinedBehaviorSanitizer in the host code;
    the process must have libasan preloaded), GFPDOT_DEBUG=1 the build with
    device-side checks."""
    global _lib
    if _lib is None:
        path = lib_path()
        if auto_build:
            _build.build(sanitize=os.environ.get("GFPDOT_SANITIZED") == "1",
                         debug=os.environ.get("GFPDOT_DEBUG") == "1")
        if not os.path.exists(path):
            raise RuntimeError(f"libgfpdot.so is missing at {path}: build it with "
                               "paper_cs_0404008_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def lib_path() -> str:
    """The library load() uses: the host-sanitized build when
    GFPDOT_SANITIZED=1, the device-checks build when GFPDOT_DEBUG=1, else the
    release build."""
    if os.environ.get("GFPDOT_SANITIZED") == "1":
        return _build.SAN_LIB
    if os.environ.get("GFPDOT_DEBUG") == "1":
        return _build.DEBUG_LIB
    return _build.LIB


def declared_symbols() -> list[str]:
    return sorted(_SIGS)


def _check(st: int, where: str):
    if st != GFP_OK:
        raise GfpError(st, where)


def _ptr(t) -> int:
    """Device (or host) address of a tensor / numpy array / int."""
    if t is None:
        return 0
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if hasattr(t, "ctypes"):
        return t.ctypes.data
    raise TypeError(f"cannot take the address of {type(t)}")


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check_u32(t, n: int, name: str):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.dtype not in (torch.uint32, torch.int32):
        raise TypeError(f"{name} must be uint32 (or int32 bit-identical), got {t.dtype}")
    if not t.is_cuda:
        raise ValueError(f"{name} must be on a CUDA device")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() < n:
        raise ValueError(f"{name} has {t.numel()} elements, needs {n}")


# ---- host-only functions ----

def gfp_status_string(st: int) -> str:
    return load().gfp_status_string(st).decode()


def gfp_delay_bound(p: int, acc_bits: int, carried: int) -> int:
    return int(load().gfp_delay_bound(p, acc_bits, carried))


def gfp_get_params(p: int) -> dict:
    out = gfp_params()
    _check(load().gfp_get_params(p, ctypes.byref(out)), "gfp_get_params")
    return {f: getattr(out, f) for f, _ in gfp_params._fields_}


def gfp_reduce_u64(x: int, p: int) -> int:
    return int(load().gfp_reduce_u64(x, p))


def gfp_reduce_f64(T: float, p: int) -> float:
    return float(load().gfp_reduce_f64(T, p))


def gfp_choose_repr(ctx, p: int, n: int) -> int:
    return int(load().gfp_choose_repr(ctx.handle if ctx else None, p, n))


# ---- context ----

class Context:
    """Owns a gfp_ctx handle bound to one CUDA device."""

    def __init__(self, device: int = 0):
        import torch
        torch.cuda.init()
        h = _vp()
        _check(load().gfp_context_create(device, ctypes.byref(h)), "gfp_context_create")
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            _check(load().gfp_context_destroy(self.handle), "gfp_context_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_repr(self, repr_: int):
        _check(load().gfp_set_repr(self.handle, repr_), "gfp_set_repr")

    def set_validate(self, on: bool):
        _check(load().gfp_set_validate(self.handle, int(bool(on))), "gfp_set_validate")

    def launch_count(self) -> int:
        return int(load().gfp_launch_count(self.handle))


def gfp_context_create(device: int = 0) -> Context:
    return Context(device)


def gfp_context_destroy(ctx: Context):
    ctx.close()


def gfp_set_repr(ctx: Context, repr_: int):
    ctx.set_repr(repr_)


def gfp_set_validate(ctx: Context, on: bool):
    ctx.set_validate(on)


def gfp_launch_count(ctx: Context) -> int:
    return ctx.launch_count()


# ---- dot products ----

def gfp_dot(ctx: Context, p: int, x, y, out, stream=None, n: int | None = None):
    """out[0] = dot(x[:n], y[:n]) mod p (device tensors)."""
    n = x.numel() if n is None else n
    _check_u32(x, n, "x")
    _check_u32(y, n, "y")
    _check_u32(out, 1, "out")
    _check(load().gfp_dot(ctx.handle, p, n, _ptr(x), _ptr(y), _ptr(out), _stream(stream)),
           "gfp_dot")
    return out


def _descs(pairs):
    """pairs: iterable of (p, x, y[, n[, repr]]) with x, y device tensors or raw addresses."""
    pairs = list(pairs)
    arr = (gfp_dot_desc * max(1, len(pairs)))()
    for j, t in enumerate(pairs):
        p, x, y = t[0], t[1], t[2]
        n = t[3] if len(t) > 3 and t[3] is not None else x.numel()
        r = t[4] if len(t) > 4 else GFP_REPR_AUTO
        arr[j].p = p
        arr[j].repr = r
        arr[j].n = n
        arr[j].x = _ptr(x)
        arr[j].y = _ptr(y)
    return arr, len(pairs)


def gfp_dot_batched(ctx: Context, pairs, out, stream=None):
    arr, count = _descs(pairs)
    if count:
        _check_u32(out, count, "out")
    _check(load().gfp_dot_batched(ctx.handle, arr, count, _ptr(out), _stream(stream)),
           "gfp_dot_batched")
    return out


def gfp_dot_batched_noalloc(pairs, out, stream=None):
    """Batched dot products using the library's fixed device scratch array
    (no allocation anywhere; at most 1024 pairs, see the header)."""
    arr, count = _descs(pairs)
    if count:
        _check_u32(out, count, "out")
    _check(load().gfp_dot_batched_noalloc(arr, count, _ptr(out), _stream(stream)),
           "gfp_dot_batched_noalloc")
    return out


class BatchPlan:
    """gfp_batch_plan: device-resident work list, one launch per exec."""

    def __init__(self, ctx: Context, pairs):
        arr, count = _descs(pairs)
        h = _vp()
        _check(load().gfp_batch_plan_create(ctx.handle, arr, count, ctypes.byref(h)),
               "gfp_batch_plan_create")
        self.handle = h
        self.count = count
        self._keep = pairs  # keep operand tensors alive with the plan

    def exec(self, out, stream=None):
        _check_u32(out, self.count, "out")
        _check(load().gfp_batch_plan_exec(self.handle, _ptr(out), _stream(stream)),
               "gfp_batch_plan_exec")
        return out

    def info(self):
        u, b = _u64(), _u64()
        _check(load().gfp_batch_plan_info(self.handle, ctypes.byref(u), ctypes.byref(b)),
               "gfp_batch_plan_info")
        return int(u.value), int(b.value)

    def close(self):
        if self.handle:
            load().gfp_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gfp_batch_plan_create(ctx: Context, pairs) -> BatchPlan:
    return BatchPlan(ctx, pairs)


def gfp_batch_plan_exec(plan: BatchPlan, out, stream=None):
    return plan.exec(out, stream)


def gfp_batch_plan_destroy(plan: BatchPlan):
    plan.close()


def gfp_dot_batched_host(ctx: Context, ps, ns, offs, x_host, y_host, out_host, stream=None):
    """Host-buffer batch (numpy or pinned CPU tensors); synchronous."""
    import numpy as np
    ps = np.ascontiguousarray(ps, dtype=np.uint32)
    ns = np.ascontiguousarray(ns, dtype=np.uint64)
    offs = np.ascontiguousarray(offs, dtype=np.uint64)
    total = int(x_host.numel() if hasattr(x_host, "numel") else x_host.shape[0])
    _check(load().gfp_dot_batched_host(ctx.handle, ps.shape[0], ps.ctypes.data, ns.ctypes.data,
                                       offs.ctypes.data, _ptr(x_host), _ptr(y_host), total,
                                       _ptr(out_host), _stream(stream)),
           "gfp_dot_batched_host")
    return out_host


# ---- matrix-vector ----

def gfp_matvec(ctx: Context, p: int, A, x, y, stream=None, lda: int | None = None,
               rows: int | None = None, cols: int | None = None):
    rows = A.shape[0] if rows is None else rows
    cols = A.shape[1] if cols is None else cols
    lda = A.stride(0) if lda is None else lda
    _check_u32(x, cols, "x")
    _check_u32(y, rows, "y")
    _check(load().gfp_matvec(ctx.handle, p, rows, cols, _ptr(A), lda, _ptr(x), _ptr(y),
                             _stream(stream)), "gfp_matvec")
    return y


def gfp_matvec_iterate(ctx: Context, p: int, A, x0, Y, iters: int, stream=None,
                       lda: int | None = None):
    n = A.shape[0]
    lda = A.stride(0) if lda is None else lda
    _check_u32(x0, n, "x0")
    _check_u32(Y, n * iters, "Y")
    _check(load().gfp_matvec_iterate(ctx.handle, p, n, _ptr(A), lda, _ptr(x0), _ptr(Y), iters,
                                     _stream(stream)), "gfp_matvec_iterate")
    return Y


def gfp_matvec_sequence(ctx: Context, p: int, A, x0, u, seq, iters: int, Y=None, stream=None,
                        lda: int | None = None):
    """seq[t] = u^T A^t x0 mod p, t = 0..iters (device tensors)."""
    n = A.shape[0]
    lda = A.stride(0) if lda is None else lda
    _check_u32(x0, n, "x0")
    _check_u32(u, n, "u")
    _check_u32(seq, iters + 1, "seq")
    if Y is not None:
        _check_u32(Y, n * iters, "Y")
    _check(load().gfp_matvec_sequence(ctx.handle, p, n, _ptr(A), lda, _ptr(x0), _ptr(u), iters,
                                      _ptr(seq), _ptr(Y), _stream(stream)), "gfp_matvec_sequence")
    return seq


# ---- block products ----

def gfp_matmul_block(ctx: Context, p: int, A, B, C, stream=None):
    """C = A B mod p for 2-D device tensors (row strides become lda/ldb/ldc)."""
    m, k = A.shape
    k2, nb = B.shape
    if k2 != k or tuple(C.shape) != (m, nb):
        raise ValueError("shape mismatch")
    for t, name in ((A, "A"), (B, "B"), (C, "C")):
        if t.dtype.itemsize != 4 or t.stride(1) != 1:
            raise ValueError(f"{name} must be a row-major 32-bit matrix")
    _check(load().gfp_matmul_block(ctx.handle, p, m, k, nb, _ptr(A), A.stride(0), _ptr(B),
                                   B.stride(0), _ptr(C), C.stride(0), _stream(stream)),
           "gfp_matmul_block")
    return C


class BlockPrep:
    """gfp_block_prep: A prepared once (tensor-core digit images) for repeated
    block products with the same A."""

    def __init__(self, ctx: Context, p: int, A):
        m, k = A.shape
        if A.dtype.itemsize != 4 or A.stride(1) != 1:
            raise ValueError("A must be a row-major 32-bit matrix")
        h = _vp()
        _check(load().gfp_block_prepare(ctx.handle, p, m, k, _ptr(A), A.stride(0), ctypes.byref(h)),
               "gfp_block_prepare")
        self.handle, self.p, self.m, self.k = h, p, m, k

    def info(self):
        b, n = _u64(), _u32()
        _check(load().gfp_block_prep_info(self.handle, ctypes.byref(b), ctypes.byref(n)),
               "gfp_block_prep_info")
        return int(b.value), int(n.value)

    def matmul(self, ctx: Context, B, C, stream=None):
        k2, nb = B.shape
        if k2 != self.k or tuple(C.shape) != (self.m, nb):
            raise ValueError("shape mismatch")
        for t, name in ((B, "B"), (C, "C")):
            if t.dtype.itemsize != 4 or t.stride(1) != 1:
                raise ValueError(f"{name} must be a row-major 32-bit matrix")
        _check(load().gfp_matmul_block_prepared(ctx.handle, self.handle, nb, _ptr(B), B.stride(0),
                                                _ptr(C), C.stride(0), _stream(stream)),
               "gfp_matmul_block_prepared")
        return C

    def close(self):
        if self.handle:
            _check(load().gfp_block_prep_destroy(self.handle), "gfp_block_prep_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gfp_block_prepare(ctx: Context, p: int, A) -> BlockPrep:
    return BlockPrep(ctx, p, A)


def gfp_matmul_block_prepared(ctx: Context, prep: BlockPrep, B, C, stream=None):
    return prep.matmul(ctx, B, C, stream)


def gfp_block_prep_info(prep: BlockPrep):
    return prep.info()


def gfp_block_prep_destroy(prep: BlockPrep):
    prep.close()


def gfp_matmul_block_csr(ctx: Context, p: int, k: int, row_ptr, col, val, B, C, stream=None):
    m = row_ptr.numel() - 1
    k2, nb = B.shape
    if k2 != k or tuple(C.shape) != (m, nb):
        raise ValueError("shape mismatch")
    _check(load().gfp_matmul_block_csr(ctx.handle, p, m, k, nb, _ptr(row_ptr), _ptr(col), _ptr(val),
                                       _ptr(B), B.stride(0), _ptr(C), C.stride(0), _stream(stream)),
           "gfp_matmul_block_csr")
    return C


def gfp_context_check(ctx: Context) -> int:
    """Synchronise; returns the status (GFP_OK, GFP_ERR_TIMEOUT, GFP_ERR_CUDA)."""
    return int(load().gfp_context_check(ctx.handle))


def gfp_wait_selftest(limit_ns: int, stream=None) -> int:
    """Returns the status (GFP_ERR_TIMEOUT expected: the bounded wait expired)."""
    return int(load().gfp_wait_selftest(limit_ns, _stream(stream)))


# ---- tuning ----

def gfp_tune(ctx: Context, primes=None, lg_lo: int = 8, lg_hi: int = 20,
             plan_path: str | None = None):
    import numpy as np
    arr = None if primes is None else np.ascontiguousarray(primes, dtype=np.uint32)
    _check(load().gfp_tune(ctx.handle, None if arr is None else arr.ctypes.data,
                           0 if arr is None else arr.shape[0], lg_lo, lg_hi,
                           plan_path.encode() if plan_path else None), "gfp_tune")


def gfp_plan_load(ctx: Context, path: str):
    _check(load().gfp_plan_load(ctx.handle, path.encode()), "gfp_plan_load")


def gfp_plan_save(ctx: Context, path: str):
    _check(load().gfp_plan_save(ctx.handle, path.encode()), "gfp_plan_save")


def gfp_plan_size(ctx: Context) -> int:
    return int(load().gfp_plan_size(ctx.handle))


# ---- synthetic inputs ----

def gfp_fill_uniform(p: int, seed: int, stream_id: int, out, n: int | None = None,
                     offset: int = 0, stream=None):
    n = out.numel() if n is None else n
    _check_u32(out, n, "out")
    _check(load().gfp_fill_uniform(p, seed, stream_id, offset, n, _ptr(out), _stream(stream)),
           "gfp_fill_uniform")
    return out


# ---- finite fields GF(p^k), discrete-logarithm representation ----

def gfp_gfq_find_primitive(p: int, k: int):
    import numpy as np
    f = np.zeros(max(k, 1), np.uint32)
    _check(load().gfp_gfq_find_primitive(p, k, f.ctypes.data), "gfp_gfq_find_primitive")
    return f


def _check_u16(t, n: int, name: str):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.dtype not in (torch.uint16, torch.int16):
        raise TypeError(f"{name} must be uint16 (or int16 bit-identical), got {t.dtype}")
    if not t.is_cuda or not t.is_contiguous() or t.numel() < n:
        raise ValueError(f"{name} must be a contiguous CUDA tensor of >= {n} elements")


class Field:
    """gfp_gfq: GF(p^k) (q <= 2^16) in the discrete-logarithm representation."""

    def __init__(self, p: int, k: int, f, device: int = 0):
        import numpy as np
        import torch
        torch.cuda.init()
        fv = np.ascontiguousarray(f, dtype=np.uint32)
        if fv.shape != (k,):
            raise ValueError("f needs k coefficients f[0..k-1]")
        h = _vp()
        _check(load().gfp_gfq_create(device, p, k, fv.ctypes.data, ctypes.byref(h)), "gfp_gfq_create")
        self.handle = h
        self.p, self.k, self.q = p, k, p ** k

    def close(self):
        if self.handle:
            _check(load().gfp_gfq_destroy(self.handle), "gfp_gfq_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        p, k, q = _u32(), _u32(), _u32()
        _check(load().gfp_gfq_info(self.handle, ctypes.byref(p), ctypes.byref(k), ctypes.byref(q)),
               "gfp_gfq_info")
        return p.value, k.value, q.value

    def to_log(self, values, codes, n: int | None = None, stream=None):
        n = values.numel() if n is None else n
        _check_u32(values, n, "values")
        _check_u16(codes, n, "codes")
        _check(load().gfp_gfq_to_log(self.handle, n, _ptr(values), _ptr(codes), _stream(stream)),
               "gfp_gfq_to_log")
        return codes

    def from_log(self, codes, values, n: int | None = None, stream=None):
        n = codes.numel() if n is None else n
        _check_u16(codes, n, "codes")
        _check_u32(values, n, "values")
        _check(load().gfp_gfq_from_log(self.handle, n, _ptr(codes), _ptr(values), _stream(stream)),
               "gfp_gfq_from_log")
        return values

    def dot(self, x, y, out, n: int | None = None, stream=None):
        n = x.numel() if n is None else n
        _check_u16(x, n, "x")
        _check_u16(y, n, "y")
        _check_u16(out, 1, "out")
        _check(load().gfp_gfq_dot(self.handle, n, _ptr(x), _ptr(y), _ptr(out), _stream(stream)),
               "gfp_gfq_dot")
        return out

    def check(self) -> int:
        return int(load().gfp_gfq_check(self.handle))


# ---- service ----

class Server:
    """gfp_server: continuous batching of dot / matvec / block jobs."""

    def __init__(self, device: int = 0, mem_budget: int = 0, max_inflight: int = 0,
                 n_streams: int = 0, queue_capacity: int = 0, batch_window_us: int = 0,
                 simulate: bool = False, fail_every: int = 0, block_sm_percent: int = 0):
        if not simulate:
            import torch
            torch.cuda.init()
        cfg = gfp_server_cfg(device, mem_budget, max_inflight, n_streams, queue_capacity,
                             batch_window_us, int(bool(simulate)), fail_every, block_sm_percent)
        h = _vp()
        _check(load().gfp_server_create(ctypes.byref(cfg), ctypes.byref(h)), "gfp_server_create")
        self.handle = h

    def close(self):
        if self.handle:
            _check(load().gfp_server_destroy(self.handle), "gfp_server_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def register_matrix(self, p: int, rows: int, cols: int, dev=None, seed: int = 0) -> int:
        h = _u64()
        _check(load().gfp_register_matrix(self.handle, p, rows, cols, _ptr(dev), seed,
                                          ctypes.byref(h)), "gfp_register_matrix")
        return int(h.value)

    def prepare_matrix(self, handle: int):
        """Build the block-product digit images of a registered matrix now."""
        _check(load().gfp_prepare_matrix(self.handle, handle), "gfp_prepare_matrix")

    def submit_status(self, kind: int, p: int, n: int = 0, nb: int = 0, matrix: int = 0,
                      x=None, y=None, v=None, seed: int = 0):
        """Returns (status, ticket) without raising."""
        j = gfp_job(kind, p, n, nb, matrix, _ptr(x), _ptr(y), _ptr(v), seed)
        t = _u64()
        st = load().gfp_submit(self.handle, ctypes.byref(j), ctypes.byref(t))
        return st, int(t.value)

    def submit(self, *a, **k) -> int:
        st, t = self.submit_status(*a, **k)
        _check(st, "gfp_submit")
        return t

    def poll(self, ticket: int):
        r = gfp_result()
        st = load().gfp_poll(self.handle, ticket, ctypes.byref(r))
        return st, r

    def wait(self, ticket: int, timeout_us: int = 60_000_000):
        r = gfp_result()
        st = load().gfp_wait(self.handle, ticket, timeout_us, ctypes.byref(r))
        return st, r

    def result_copy(self, ticket: int, count: int):
        import numpy as np
        out = np.zeros(count, dtype=np.uint32)
        _check(load().gfp_result_copy(self.handle, ticket, out.ctypes.data, count),
               "gfp_result_copy")
        return out

    def release(self, ticket: int) -> int:
        return int(load().gfp_release(self.handle, ticket))

    def stats(self) -> dict:
        s = gfp_server_stats()
        _check(load().gfp_server_get_stats(self.handle, ctypes.byref(s)), "gfp_server_get_stats")
        return {f: getattr(s, f) for f, _ in gfp_server_stats._fields_}


def gfp_server_create(**kw) -> Server:
    return Server(**kw)


def gfp_server_destroy(srv: Server):
    srv.close()
