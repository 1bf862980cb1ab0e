"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module holds input synthesis only: it performs none of the field
arithmetic that the dot-product method computes.  Both the oracle tests and
the GPU path draw their operands from here, so the two sides agree on inputs
without sharing any of the method's code.

Generator
---------
Counter-based SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; the finaliser constants are the
published ones of that paper's `mix64` variant as popularised by Vigna's
public-domain ``splitmix64.c``)::

    mix64(z)     = z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
                   z ^= z >> 27; z *= 0x94D049BB133111EB; z ^ (z >> 31)
    key(s, t)    = mix64(s + GAMMA * (t + 1))          (mod 2^64)
    word(s,t,i)  = mix64(key(s, t) + GAMMA * (i + 1))  (mod 2^64)
    residue      = word mod p                          (bias < p / 2^64)

with GAMMA = 0x9E3779B97F4A7C15.  ``s`` is the seed, ``t`` a stream number
(one per vector) and ``i`` the element index, so any element can be
regenerated independently (the device generator in the library implements the
same definition and is checked against this one).

Workload shapes follow the paper's experiments (random vectors of residues
modulo word-size primes, Section 2.5 and Section 3) scaled to the sizes of the
five benchmark workloads described in the design notes.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1

#: Primes of the benchmark workloads (the paper's 32749 of Section 2.5, the
#: largest primes below 2^16, 2^26 and 2^32, and the Mersenne prime 2^31-1).
PRIMES_BATCHED = (32749, 65521, 67108859, 2147483647, 4294967291)
PRIMES_SERVE = (65521, 67108859, 4294967291)

#: Base seed of the synthetic workloads; workload c uses BASE_SEED + c.
BASE_SEED = 0x0404008


def _mix64_inplace(z: np.ndarray) -> np.ndarray:
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def mix64_int(z: int) -> int:
    """Scalar SplitMix64 finaliser on a Python int (for keys and tests)."""
    z &= _MASK64
    z ^= z >> 30
    z = (z * 0xBF58476D1CE4E5B9) & _MASK64
    z ^= z >> 27
    z = (z * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def stream_key(seed: int, stream: int) -> int:
    return mix64_int((seed + 0x9E3779B97F4A7C15 * (stream + 1)) & _MASK64)


def words(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Raw 64-bit words ``word(seed, stream, offset .. offset+n-1)``."""
    key = np.uint64(stream_key(seed, stream))
    idx = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = idx * GAMMA
        z += key
        return _mix64_inplace(z)


_CHUNK = 1 << 22


def _uniform_into(out: np.ndarray, p: int, seed: int, stream: int, offset: int) -> None:
    w = words(seed, stream, out.shape[0], offset)
    out[:] = (w % np.uint64(p)).astype(np.uint32)


def uniform(p: int, n: int, seed: int, stream: int, offset: int = 0,
            threads: int | None = None) -> np.ndarray:
    """n residues uniform in [0, p) as uint32 (chunked over host threads)."""
    if not 2 <= p <= 0xFFFFFFFF:
        raise ValueError("p must be in [2, 2^32-1]")
    out = np.empty(n, dtype=np.uint32)
    if n <= _CHUNK:
        if n:
            _uniform_into(out, p, seed, stream, offset)
        return out
    nth = threads or max(1, min(16, len(os.sched_getaffinity(0))))
    starts = range(0, n, _CHUNK)
    with ThreadPoolExecutor(nth) as ex:
        list(ex.map(lambda s: _uniform_into(out[s:s + _CHUNK], p, seed, stream, offset + s),
                    starts))
    return out


def unit_doubles(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles uniform in [0, 1) from the top 53 bits of the words."""
    w = words(seed, stream, n)
    return (w >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


# --------------------------------------------------------------------------
# Workload recipes
# --------------------------------------------------------------------------

def batched_shapes(count: int, seed: int, lg_lo: float = 8.0, lg_hi: float = 20.0,
                   primes=PRIMES_BATCHED):
    """Lengths floor(2^U), U ~ Uniform(lg_lo, lg_hi), and primes uniform over
    ``primes`` for ``count`` pairs (stream 0 = lengths, stream 1 = primes)."""
    u = unit_doubles(seed, 0, count)
    lens = np.floor(np.exp2(lg_lo + (lg_hi - lg_lo) * u)).astype(np.int64)
    pw = words(seed, 1, count)
    pidx = (pw % np.uint64(len(primes))).astype(np.int64)
    ps = np.asarray(primes, dtype=np.int64)[pidx]
    return lens, ps


def aligned_offsets(lens: np.ndarray, align: int = 4) -> tuple[np.ndarray, int]:
    """Element offsets packing vectors back to back, each start a multiple
    of ``align`` elements (16 bytes for align=4); returns (offsets, total)."""
    padded = (lens + (align - 1)) // align * align
    off = np.zeros(len(lens), dtype=np.int64)
    if len(lens) > 1:
        off[1:] = np.cumsum(padded)[:-1]
    total = int(padded.sum())
    return off, total


def batched_operands(lens, ps, seed: int):
    """Packed x and y host buffers for a batch: pair i occupies
    [off[i], off[i]+lens[i]) of each buffer; x uses stream 2+2i, y 3+2i."""
    off, total = aligned_offsets(np.asarray(lens))
    x = np.zeros(total, dtype=np.uint32)
    y = np.zeros(total, dtype=np.uint32)
    for i, (n, p) in enumerate(zip(lens, ps)):
        n = int(n)
        if n:
            x[off[i]:off[i] + n] = uniform(int(p), n, seed, 2 + 2 * i)
            y[off[i]:off[i] + n] = uniform(int(p), n, seed, 3 + 2 * i)
    return off, total, x, y


def expected_total_macs(count: int, lg_lo: float = 8.0, lg_hi: float = 20.0) -> float:
    """E[sum of lengths] for log-uniform lengths (continuous approximation)."""
    return count * (2.0 ** lg_hi - 2.0 ** lg_lo) / ((lg_hi - lg_lo) * math.log(2.0))


def csr_pattern(m: int, k: int, density: float, p: int, seed: int):
    """Bernoulli(density) sparsity per row at uniform columns, values uniform
    in [1, p): returns row_ptr (uint32[m+1]), col (uint32[nnz]), val (uint32[nnz])."""
    rows_col = []
    rows_val = []
    row_ptr = np.zeros(m + 1, dtype=np.uint32)
    for i in range(m):
        u = unit_doubles(seed, 4 * i + 0, k)
        cols = np.nonzero(u < density)[0].astype(np.uint32)
        vals = (uniform(p - 1, len(cols), seed, 4 * i + 1) + 1).astype(np.uint32) if len(cols) else cols
        rows_col.append(cols)
        rows_val.append(vals)
        row_ptr[i + 1] = row_ptr[i] + len(cols)
    col = np.concatenate(rows_col) if rows_col else np.zeros(0, np.uint32)
    val = np.concatenate(rows_val) if rows_val else np.zeros(0, np.uint32)
    return row_ptr, col.astype(np.uint32), val.astype(np.uint32)


def serve_requests(count: int, seed: int):
    """Seeded request mix of the serving workload: 70% dot (n log-uniform
    [2^10, 2^22], p uniform over PRIMES_SERVE), 25% matrix-vector and 5% block
    jobs over pools of 16 registered matrices per kind (see serve_pool_specs).
    Request i is (kind, p or None, n, pool index, job seed); kind 0 dot,
    1 matrix-vector, 2 block.  The first c requests of a longer stream are the
    requests of serve_requests(c, seed)."""
    u = unit_doubles(seed, 10, count)
    v = unit_doubles(seed, 11, count)
    w = words(seed, 12, count)
    kinds = np.where(u < 0.70, 0, np.where(u < 0.95, 1, 2))
    reqs = []
    for i in range(count):
        k = int(kinds[i])
        if k == 0:
            n = int(np.floor(2.0 ** (10 + 12 * v[i])))
            reqs.append((0, PRIMES_SERVE[int(w[i] % np.uint64(3))], n, 0, seed * 1000003 + i))
        else:
            reqs.append((k, None, 0, int(w[i] % np.uint64(16)), seed * 1000003 + i))
    return reqs


def serve_pool_specs(seed: int):
    """The registered matrices of the serving workload: for kind 1
    (matrix-vector) 16 square matrices with side log-uniform [2^10, 2^14], for
    kind 2 (block, nb = 64) 16 with side log-uniform [2^10, 2^13]; p uniform
    over PRIMES_SERVE.  Returns {kind: [(p, side, matrix seed)] * 16}; matrix
    entries are uniform(p, side*side, matrix seed, 0) in row-major order."""
    pools = {1: [], 2: []}
    for kind, lo, hi in ((1, 10, 14), (2, 10, 13)):
        du = unit_doubles(seed, 20 + kind, 16)
        dw = words(seed, 22 + kind, 16)
        for i in range(16):
            side = int(np.floor(2.0 ** (lo + (hi - lo) * du[i])))
            p = PRIMES_SERVE[int(dw[i] % np.uint64(3))]
            pools[kind].append((p, side, seed * 7919 + kind * 100 + i))
    return pools
