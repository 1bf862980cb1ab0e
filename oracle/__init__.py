"""CPU oracle for the exact GF(p) dot product and its derived products.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by
the CPU-baseline leg of the benchmark, never by the library.  It shares no code
with the CUDA path; the C source is ``gfp_oracle.c`` in this directory (per
term Zpz arithmetic, Section 2.1 of the paper), compiled with the host C
compiler by :func:`build` into ``oracle/_build/liboracle.so``.

All entry points take numpy uint32 arrays of canonical residues (< p).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gfp_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

_lib = None
_lock = threading.Lock()

_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain -O2, no -march)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"],
                       check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def bind(lib):
    """Declare the C signatures on a loaded oracle library (used for the
    default build and, by the tests, for deliberately broken variants)."""
    lib.oracle_dot.restype = ctypes.c_uint32
    lib.oracle_dot.argtypes = [ctypes.c_uint32, ctypes.c_uint64, _u32p, _u32p]
    lib.oracle_dot_batch.restype = None
    lib.oracle_dot_batch.argtypes = [ctypes.c_uint64, _u32p, _u64p, _u64p, _u32p, _u32p, _u32p]
    lib.oracle_matvec_rows.restype = None
    lib.oracle_matvec_rows.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.c_uint64, _u32p, ctypes.c_uint64, _u32p, _u32p]
    lib.oracle_block_rows.restype = None
    lib.oracle_block_rows.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                      ctypes.c_uint64, ctypes.c_uint64, _u32p, ctypes.c_uint64,
                                      _u32p, ctypes.c_uint64, _u32p, ctypes.c_uint64]
    lib.oracle_csr_rows.restype = None
    lib.oracle_csr_rows.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                    ctypes.c_uint64, _u32p, _u32p, _u32p, _u32p, ctypes.c_uint64,
                                    _u32p, ctypes.c_uint64]
    lib.oracle_paper_block_dot.restype = ctypes.c_uint64
    lib.oracle_paper_block_dot.argtypes = [ctypes.c_uint32, ctypes.c_uint64, _u32p, _u32p,
                                           ctypes.c_uint64, ctypes.c_int]
    lib.oracle_paper_overflow_dot.restype = ctypes.c_uint32
    lib.oracle_paper_overflow_dot.argtypes = [ctypes.c_uint32, ctypes.c_uint64, _u32p, _u32p]
    lib.oracle_paper_fp_reduce.restype = ctypes.c_double
    lib.oracle_paper_fp_reduce.argtypes = [ctypes.c_double, ctypes.c_double]
    lib.oracle_paper_fp_dot.restype = ctypes.c_uint32
    lib.oracle_paper_fp_dot.argtypes = [ctypes.c_uint32, ctypes.c_uint64, _u32p, _u32p,
                                        ctypes.c_uint64]
    lib.oracle_gfq_add.restype = ctypes.c_uint32
    lib.oracle_gfq_add.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                   ctypes.c_uint32]
    lib.oracle_gfq_mul.restype = ctypes.c_uint32
    lib.oracle_gfq_mul.argtypes = [ctypes.c_uint32, ctypes.c_uint32, _u32p, ctypes.c_uint32,
                                   ctypes.c_uint32]
    lib.oracle_gfq_dot.restype = ctypes.c_uint32
    lib.oracle_gfq_dot.argtypes = [ctypes.c_uint32, ctypes.c_uint32, _u32p, ctypes.c_uint64,
                                   _u32p, _u32p]
    return lib


def compile_variant(source: str, out_dir: str, name: str):
    """Compile an edited copy of the oracle source (tests plant mistakes in
    copies to check that the pins catch them) and return the bound library."""
    src = os.path.join(out_dir, name + ".c")
    so = os.path.join(out_dir, name + ".so")
    with open(src, "w") as f:
        f.write(source)
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", so, src, "-lm"], check=True)
    return bind(ctypes.CDLL(so))


def source() -> str:
    with open(_SRC) as f:
        return f.read()


_override = threading.local()


class use:
    """Context manager: route this thread's oracle calls to another bound
    library (a planted-mistake variant in the tests)."""

    def __init__(self, lib):
        self.lib = lib

    def __enter__(self):
        self.prev = getattr(_override, "lib", None)
        _override.lib = self.lib
        return self

    def __exit__(self, *exc):
        _override.lib = self.prev


def _load():
    global _lib
    ov = getattr(_override, "lib", None)
    if ov is not None:
        return ov
    with _lock:
        if _lib is None:
            _lib = bind(ctypes.CDLL(build()))
    return _lib


def _p32(a: np.ndarray):
    assert a.dtype == np.uint32 and a.flags.c_contiguous
    return a.ctypes.data_as(_u32p)


def _p64(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags.c_contiguous
    return a.ctypes.data_as(_u64p)


def _threads(n: int | None) -> int:
    return n or max(1, len(os.sched_getaffinity(0)))


def dot(p: int, x: np.ndarray, y: np.ndarray) -> int:
    """(sum x_i*y_i) mod p, term by term."""
    x = np.ascontiguousarray(x, dtype=np.uint32)
    y = np.ascontiguousarray(y, dtype=np.uint32)
    assert x.shape == y.shape
    return int(_load().oracle_dot(p, x.shape[0], _p32(x), _p32(y)))


def dot_batch(ps, lens, offs, x: np.ndarray, y: np.ndarray, threads: int | None = None):
    """Residues of packed pairs (pair j at offs[j], length lens[j], prime ps[j])."""
    lib = _load()
    ps = np.ascontiguousarray(ps, dtype=np.uint32)
    lens = np.ascontiguousarray(lens, dtype=np.uint64)
    offs = np.ascontiguousarray(offs, dtype=np.uint64)
    x = np.ascontiguousarray(x, dtype=np.uint32)
    y = np.ascontiguousarray(y, dtype=np.uint32)
    count = ps.shape[0]
    out = np.zeros(count, dtype=np.uint32)
    nth = _threads(threads)
    # split pairs into nth contiguous groups of similar total length
    bounds = np.searchsorted(np.cumsum(lens.astype(np.float64)),
                             np.linspace(0, float(lens.sum()), nth + 1)[1:-1])
    edges = [0] + [int(b) for b in bounds] + [count]

    def run(g):
        a, b = edges[g], edges[g + 1]
        if b > a:
            lib.oracle_dot_batch(b - a, _p32(ps[a:b]), _p64(lens[a:b]), _p64(offs[a:b]),
                                 _p32(x), _p32(y), _p32(out[a:b]))
    with ThreadPoolExecutor(nth) as ex:
        list(ex.map(run, range(len(edges) - 1)))
    return out


def _row_split(rows: int, nth: int):
    step = max(1, -(-rows // nth))
    return [(r, min(rows, r + step)) for r in range(0, rows, step)]


def matvec(p: int, A: np.ndarray, x: np.ndarray, rows: range | None = None,
           threads: int | None = None) -> np.ndarray:
    """y = A x mod p for a row-major uint32 matrix (all rows, or ``rows``)."""
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.uint32)
    x = np.ascontiguousarray(x, dtype=np.uint32)
    m, k = A.shape
    assert x.shape == (k,)
    y = np.zeros(m, dtype=np.uint32)
    r0, r1 = (0, m) if rows is None else (rows.start, rows.stop)

    def run(rr):
        lib.oracle_matvec_rows(p, rr[0], rr[1], k, _p32(A), k, _p32(x), _p32(y))
    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(run, [(r0 + a, r0 + b) for a, b in _row_split(r1 - r0, _threads(threads))]))
    return y


def block(p: int, A: np.ndarray, B: np.ndarray, threads: int | None = None) -> np.ndarray:
    """C = A B mod p, A m x k and B k x nb row-major uint32."""
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.uint32)
    B = np.ascontiguousarray(B, dtype=np.uint32)
    m, k = A.shape
    k2, nb = B.shape
    assert k == k2
    C = np.zeros((m, nb), dtype=np.uint32)

    def run(rr):
        lib.oracle_block_rows(p, rr[0], rr[1], k, nb, _p32(A), k, _p32(B), nb, _p32(C), nb)
    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(run, _row_split(m, _threads(threads))))
    return C


def block_rows(p: int, A: np.ndarray, B: np.ndarray, rows) -> np.ndarray:
    """Selected rows of A B mod p (rows: iterable of row indices)."""
    rows = np.asarray(list(rows), dtype=np.int64)
    return block(p, np.ascontiguousarray(A[rows]), B, threads=1)


def csr(p: int, row_ptr, col, val, B: np.ndarray, threads: int | None = None) -> np.ndarray:
    """C = A B mod p for a CSR matrix A (row_ptr, col, val) and dense B."""
    lib = _load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.uint32)
    col = np.ascontiguousarray(col, dtype=np.uint32)
    val = np.ascontiguousarray(val, dtype=np.uint32)
    B = np.ascontiguousarray(B, dtype=np.uint32)
    m = row_ptr.shape[0] - 1
    nb = B.shape[1]
    C = np.zeros((m, nb), dtype=np.uint32)
    if col.shape[0] == 0:
        col = np.zeros(1, np.uint32)
        val = np.zeros(1, np.uint32)

    def run(rr):
        lib.oracle_csr_rows(p, rr[0], rr[1], nb, _p32(row_ptr), _p32(col), _p32(val), _p32(B),
                            nb, _p32(C), nb)
    with ThreadPoolExecutor(_threads(threads)) as ex:
        list(ex.map(run, _row_split(m, _threads(threads))))
    return C


# ---- the paper's variants, restated (Sections 2.3, 3.1-3.3) ----

def paper_block_dot(p: int, x, y, K: int, acc_bits: int = 64):
    x = np.ascontiguousarray(x, dtype=np.uint32)
    y = np.ascontiguousarray(y, dtype=np.uint32)
    r = int(_load().oracle_paper_block_dot(p, x.shape[0], _p32(x), _p32(y), K, acc_bits))
    return None if r == (1 << 64) - 1 else r


def paper_overflow_dot(p: int, x, y) -> int:
    x = np.ascontiguousarray(x, dtype=np.uint32)
    y = np.ascontiguousarray(y, dtype=np.uint32)
    return int(_load().oracle_paper_overflow_dot(p, x.shape[0], _p32(x), _p32(y)))


def paper_fp_reduce(T: float, P: float) -> float:
    return float(_load().oracle_paper_fp_reduce(T, P))


def paper_fp_dot(p: int, x, y, K: int):
    x = np.ascontiguousarray(x, dtype=np.uint32)
    y = np.ascontiguousarray(y, dtype=np.uint32)
    r = int(_load().oracle_paper_fp_dot(p, x.shape[0], _p32(x), _p32(y), K))
    return None if r == 0xFFFFFFFF else r


# ---- finite fields GF(p^k) (Section 2.4: discrete logarithms, extensions) ----
#
# Elements are encoded as sum_j c_j p^j (c_j the coefficient of x^j) in
# GF(p)[x]/(f), f = x^k + f[k-1] x^(k-1) + ... + f[0] monic, given by f[0..k-1].

def _fvec(f, k):
    f = np.ascontiguousarray(f, dtype=np.uint32)
    assert f.shape == (k,)
    return f


def gfq_add(p: int, k: int, a: int, b: int) -> int:
    return int(_load().oracle_gfq_add(p, k, a, b))


def gfq_mul(p: int, k: int, f, a: int, b: int) -> int:
    return int(_load().oracle_gfq_mul(p, k, _p32(_fvec(f, k)), a, b))


def gfq_dot(p: int, k: int, f, x, y, threads: int = 1) -> int:
    """Field dot product sum_i x_i y_i in GF(p)[x]/(f), term by term; with
    threads > 1 the terms are split into contiguous chunks whose sums are
    added with the field addition (addition is associative and commutative)."""
    x = np.ascontiguousarray(x, dtype=np.uint32)
    y = np.ascontiguousarray(y, dtype=np.uint32)
    assert x.shape == y.shape
    lib = _load()
    fv = _fvec(f, k)
    n = x.shape[0]
    nth = max(1, min(_threads(None) if threads == 0 else threads, n // 4096 or 1))
    if nth == 1:
        return int(lib.oracle_gfq_dot(p, k, _p32(fv), n, _p32(x), _p32(y)))
    edges = np.linspace(0, n, nth + 1).astype(np.int64)

    def run(g):
        a, b = int(edges[g]), int(edges[g + 1])
        return int(lib.oracle_gfq_dot(p, k, _p32(fv), b - a, _p32(x[a:b]), _p32(y[a:b])))
    with ThreadPoolExecutor(nth) as ex:
        parts = list(ex.map(run, range(nth)))
    r = 0
    for v in parts:
        r = gfq_add(p, k, r, v)
    return r


def gfq_pow(p: int, k: int, f, a: int, e: int) -> int:
    r, b = (1 if k >= 1 else 0), a
    while e:
        if e & 1:
            r = gfq_mul(p, k, f, r, b)
        b = gfq_mul(p, k, f, b, b)
        e >>= 1
    return r


def _prime_factors(n: int):
    out, d = [], 2
    while d * d <= n:
        if n % d == 0:
            out.append(d)
            while n % d == 0:
                n //= d
        d += 1
    if n > 1:
        out.append(n)
    return out


def gfq_x_is_primitive(p: int, k: int, f) -> bool:
    """True when x generates the multiplicative group of GF(p)[x]/(f) (so the
    quotient is a field and f is a primitive polynomial)."""
    q = p ** k
    x = p if k > 1 else (p - int(f[0])) % p   # the class of x: for k = 1, x = -f[0]
    if gfq_pow(p, k, f, x, q - 1) != 1:
        return False
    return all(gfq_pow(p, k, f, x, (q - 1) // r) != 1 for r in _prime_factors(q - 1))


def gfq_find_primitive(p: int, k: int):
    """The first f (lexicographic in f[0..k-1], f[0] != 0) with x primitive."""
    import itertools
    for tail in itertools.product(range(p), repeat=k - 1):
        for f0 in range(1, p):
            f = [f0, *tail]
            if gfq_x_is_primitive(p, k, f):
                return np.array(f, dtype=np.uint32)
    raise ValueError(f"no primitive polynomial of degree {k} over GF({p})")
