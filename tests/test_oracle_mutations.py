"""The pins catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of the oracle source (a dropped term,
a wrong index, a transposed operand, a missing reduction, a wrong
correction constant, a row offset slip, a field reduction dropped or with the
wrong sign, a reversed digit order), builds it, and checks that at least
one pin fails for it while the unmodified oracle passes them all.  The
mistakes live only in temporary copies; the oracle itself is never edited."""
import random

import numpy as np
import pytest

import gfp_inputs as gi
import oracle


def bigdot(p, x, y):
    return sum(int(a) * int(b) for a, b in zip(x, y)) % p


def pins_pass() -> bool:
    """A compact subset of the pins (brute force, closed forms, invariants)."""
    rng = random.Random(7)
    try:
        for p in (2, 7, 65521, 2147483647, 4294967291):
            for n in (0, 1, 2, 5, 33):
                x = [rng.randrange(p) for _ in range(n)]
                y = [rng.randrange(p) for _ in range(n)]
                if oracle.dot(p, np.array(x, np.uint32), np.array(y, np.uint32)) != bigdot(p, x, y):
                    return False
            v = np.full(1001, p - 1, np.uint32)
            if oracle.dot(p, v, v) != 1001 % p:
                return False
        p = 4294967291
        m, k, nb = 5, 9, 4
        A = gi.uniform(p, m * k, 3, 0).reshape(m, k)
        B = gi.uniform(p, k * nb, 3, 1).reshape(k, nb)
        C = oracle.block(p, A, B, threads=1)
        if any(int(C[i, j]) != bigdot(p, A[i], B[:, j]) for i in range(m) for j in range(nb)):
            return False
        xv = gi.uniform(p, k, 3, 2)
        if oracle.matvec(p, A, xv, threads=1).tolist() != [bigdot(p, A[i], xv) for i in range(m)]:
            return False
        row_ptr, col, val = gi.csr_pattern(6, 12, 0.4, 65521, seed=4)
        Bs = gi.uniform(65521, 12 * 3, 4, 9).reshape(12, 3)
        Cs = oracle.csr(65521, row_ptr, col, val, Bs, threads=1)
        for i in range(6):
            q = range(int(row_ptr[i]), int(row_ptr[i + 1]))
            for j in range(3):
                if int(Cs[i, j]) != sum(int(val[t]) * int(Bs[col[t], j]) for t in q) % 65521:
                    return False
        for pp, K in ((65521, 5), (4294967291, 1)):
            a = gi.uniform(pp, 777, 5, 0)
            b = gi.uniform(pp, 777, 5, 1)
            if oracle.paper_overflow_dot(pp, a, b) != bigdot(pp, a, b):
                return False
            if oracle.paper_block_dot(pp, a, b, K, 64) != bigdot(pp, a, b):
                return False
        # GF(p^k): the published GF(2^8) products and the GF(9) facts by hand
        aes = [1, 1, 0, 1, 1, 0, 0, 0]
        if (oracle.gfq_mul(2, 8, aes, 0x57, 0x83), oracle.gfq_mul(2, 8, aes, 0x57, 0x13)) != (0xC1, 0xFE):
            return False
        if oracle.gfq_add(2, 8, 0x57, 0x83) != 0xD4:
            return False
        if (oracle.gfq_mul(3, 2, [1, 0], 3, 3), oracle.gfq_mul(3, 2, [1, 0], 4, 4)) != (2, 6):
            return False
        if oracle.gfq_dot(3, 2, [1, 0], [3, 4, 5], [3, 4, 0]) != oracle.gfq_add(3, 2, 2, 6):
            return False
        return True
    except Exception:
        return False


MUTATIONS = {
    "dropped_last_term": ("for (uint64_t i = 0; i < n; ++i)\n        r = zpz_axpy(r, x[i], y[i], p);",
                          "for (uint64_t i = 0; i + 1 < n; ++i)\n        r = zpz_axpy(r, x[i], y[i], p);"),
    "wrong_index": ("r = zpz_axpy(r, x[i], y[i], p);\n    return (uint32_t)r;\n}\n\n/* Strided",
                    "r = zpz_axpy(r, x[i], y[n - 1 - i], p);\n    return (uint32_t)r;\n}\n\n/* Strided"),
    "transposed_B": ("oracle_dot_strided(p, k, A + i * lda, 1, B + j, ldb);",
                     "oracle_dot_strided(p, k, A + i * lda, 1, B + j * ldb, 1);"),
    "no_remainder": ("return (r + (uint64_t)a * (uint64_t)b) % p;",
                     "return (r + (uint64_t)a * (uint64_t)b);"),
    "wrong_corr": ("const uint64_t corr = (UINT64_MAX % p + 1) % p;",
                   "const uint64_t corr = UINT64_MAX % p;"),
    "matvec_row_slip": ("y[i] = oracle_dot(p, cols, A + i * lda, x);",
                        "y[i] = oracle_dot(p, cols, A + i * cols + (i > 0), x);"),
    "csr_col_slip": ("r = zpz_axpy(r, val[q], B[(uint64_t)col[q] * ldb + j], p);",
                     "r = zpz_axpy(r, val[q], B[(uint64_t)q * 0 + col[q] + j], p);"),
    "block_tail_skipped": ("    for (; i < n; ++i)\n        res = (res + (uint64_t)a[i] * b[i]) & mask;",
                           "    for (; i + 1 < n; ++i)\n        res = (res + (uint64_t)a[i] * b[i]) & mask;"),
    "gfq_no_reduction": ("for (uint32_t m = 2 * k - 1; m-- > k;) {",
                         "for (uint32_t m = k; m-- > k;) {"),
    "gfq_reduction_sign": ("(uint64_t)(p - f[j] % p) % p * t) % p;",
                           "(uint64_t)(f[j] % p) * t) % p;"),
    "gfq_digit_order": ("for (uint32_t j = k; j-- > 0;) v = v * p + c[j];",
                        "for (uint32_t j = 0; j < k; ++j) v = v * p + c[j];"),
    "gfq_dot_drops_term": ("for (uint64_t i = 0; i < n; ++i) r = oracle_gfq_add(",
                           "for (uint64_t i = 1; i < n; ++i) r = oracle_gfq_add("),
}


def test_unmodified_oracle_passes():
    assert pins_pass()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTATIONS[name]
    src = oracle.source()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    lib = oracle.compile_variant(src.replace(old, new), str(tmp_path), name)
    with oracle.use(lib):
        assert not pins_pass(), f"no pin caught {name}"
