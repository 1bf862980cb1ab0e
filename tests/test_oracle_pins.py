"""Pins of the CPU oracle against facts that do not come from the oracle.

Brute force in arbitrary precision (Python ints) on tiny inputs, closed forms,
and invariants of the exact dot product over GF(p) (Section 2.1 definition),
plus the paper's own dot-product variants (Sections 2.3, 3.1-3.3) restated in
the oracle and checked against the plain definition.
"""
import itertools
import os
import random

import numpy as np
import pytest

import gfp_inputs as gi
import oracle

PRIMES = [2, 3, 5, 7, 13, 251, 32749, 40009, 65521, 67108859, 2147483647, 4294967291]


def bigdot(p, x, y):
    return sum(int(a) * int(b) for a, b in zip(x, y)) % p


def test_exhaustive_small_fields():
    """Every pair of vectors for tiny p and n against brute force."""
    for p, nmax in ((2, 4), (3, 4), (5, 3), (7, 2)):
        for n in range(0, nmax + 1):
            vecs = list(itertools.product(range(p), repeat=n))
            pairs = [(a, b) for a in vecs for b in vecs]
            lens = np.full(len(pairs), n, dtype=np.uint64)
            offs = np.arange(len(pairs), dtype=np.uint64) * max(n, 1)
            x = np.array([v for a, _ in pairs for v in a] or [0], dtype=np.uint32)
            y = np.array([v for _, b in pairs for v in b] or [0], dtype=np.uint32)
            ps = np.full(len(pairs), p, dtype=np.uint32)
            got = oracle.dot_batch(ps, lens, offs, x, y, threads=2)
            want = [bigdot(p, a, b) for a, b in pairs]
            assert got.tolist() == want, (p, n)


def test_random_against_bigint():
    rng = random.Random(1234)
    for p in PRIMES:
        for n in list(range(0, 9)) + [31, 63, 64]:
            x = [rng.randrange(p) for _ in range(n)]
            y = [rng.randrange(p) for _ in range(n)]
            assert oracle.dot(p, np.array(x, np.uint32), np.array(y, np.uint32)) == bigdot(p, x, y)


@pytest.mark.parametrize("p", PRIMES)
def test_all_max_closed_form(p):
    """All-(p-1) vectors: n (p-1)^2 = n (mod p); maximises every term."""
    for n in (1, 2, 3, 17, 1000, 65537):
        v = np.full(n, p - 1, np.uint32)
        assert oracle.dot(p, v, v) == n % p


@pytest.mark.parametrize("p", [32749, 65521, 4294967291])
def test_constant_vectors(p):
    rng = random.Random(p)
    for _ in range(5):
        n = rng.randrange(1, 5000)
        c, d = rng.randrange(p), rng.randrange(p)
        x = np.full(n, c, np.uint32)
        y = np.full(n, d, np.uint32)
        assert oracle.dot(p, x, y) == (n * c * d) % p
        assert oracle.dot(p, x, x) == (n * c * c) % p


def test_unit_vectors_pick_entries():
    p = 2147483647
    x = gi.uniform(p, 97, seed=5, stream=0)
    for i in (0, 1, 50, 96):
        e = np.zeros(97, np.uint32)
        e[i] = 1
        assert oracle.dot(p, x, e) == int(x[i])
        assert oracle.dot(p, e, x) == int(x[i])


def test_bilinearity_concat_and_range():
    for p in (65521, 67108859, 4294967291):
        n = 3001
        x = gi.uniform(p, n, 7, 0)
        x2 = gi.uniform(p, n, 7, 1)
        y = gi.uniform(p, n, 7, 2)
        xs = ((x.astype(np.uint64) + x2) % p).astype(np.uint32)
        d1, d2, ds = oracle.dot(p, x, y), oracle.dot(p, x2, y), oracle.dot(p, xs, y)
        assert ds == (d1 + d2) % p
        assert 0 <= ds < p
        # concatenation
        cat = oracle.dot(p, np.concatenate([x, x2]), np.concatenate([y, y]))
        assert cat == (d1 + d2) % p
        # scaling by a constant c: dot(c x, y) = c dot(x, y)
        c = 12345 % p
        cx = ((x.astype(np.uint64) * c) % p).astype(np.uint32)
        assert oracle.dot(p, cx, y) == (c * d1) % p


def test_matvec_identity_permutation_and_bruteforce():
    p = 2147483647
    n = 37
    x = gi.uniform(p, n, 9, 0)
    assert oracle.matvec(p, np.eye(n, dtype=np.uint32), x).tolist() == x.tolist()
    perm = np.random.default_rng(1).permutation(n)
    P = np.zeros((n, n), np.uint32)
    P[np.arange(n), perm] = 1
    assert oracle.matvec(p, P, x).tolist() == x[perm].tolist()
    # non-square, brute force (catches a transposed operand)
    A = gi.uniform(p, 5 * 11, 9, 1).reshape(5, 11)
    v = gi.uniform(p, 11, 9, 2)
    want = [bigdot(p, A[i], v) for i in range(5)]
    assert oracle.matvec(p, A, v).tolist() == want


def test_block_bruteforce_nonsquare():
    for p in (65521, 4294967291):
        m, k, nb = 7, 13, 5
        A = gi.uniform(p, m * k, 11, 0).reshape(m, k)
        B = gi.uniform(p, k * nb, 11, 1).reshape(k, nb)
        C = oracle.block(p, A, B, threads=2)
        for i in range(m):
            for j in range(nb):
                assert int(C[i, j]) == bigdot(p, A[i], B[:, j])


def test_block_freivalds():
    """u^T (A B) = (u^T A) B over GF(p) (exact integer identity mod p)."""
    p = 65521
    m, k, nb = 64, 200, 16
    A = gi.uniform(p, m * k, 12, 0).reshape(m, k)
    B = gi.uniform(p, k * nb, 12, 1).reshape(k, nb)
    u = gi.uniform(p, m, 12, 2)
    C = oracle.block(p, A, B)
    lhs = [bigdot(p, u, C[:, j]) for j in range(nb)]
    uA = [bigdot(p, u, A[:, t]) for t in range(k)]
    rhs = [bigdot(p, uA, B[:, j]) for j in range(nb)]
    assert lhs == rhs


def test_csr_bruteforce():
    p = 65521
    m, k, nb = 9, 40, 6
    row_ptr, col, val = gi.csr_pattern(m, k, 0.2, p, seed=3)
    B = gi.uniform(p, k * nb, 3, 1000).reshape(k, nb)
    C = oracle.csr(p, row_ptr, col, val, B, threads=2)
    for i in range(m):
        q = range(int(row_ptr[i]), int(row_ptr[i + 1]))
        for j in range(nb):
            want = sum(int(val[t]) * int(B[col[t], j]) for t in q) % p
            assert int(C[i, j]) == want
    # empty rows give zeros
    rp0 = np.zeros(4, np.uint32)
    C0 = oracle.csr(p, rp0, np.zeros(0, np.uint32), np.zeros(0, np.uint32), B)
    assert not C0.any()


# ---- the paper's variants restated in the oracle, checked against the definition ----

@pytest.mark.parametrize("p", [13, 251, 2887, 32749, 65521, 67108859, 2147483647, 4294967291])
def test_paper_block_dot_matches(p):
    n = 1029
    x = gi.uniform(p, n, 21, 0)
    y = gi.uniform(p, n, 21, 1)
    want = oracle.dot(p, x, y)
    pm1 = p - 1
    k64 = ((1 << 64) - pm1 - 1) // (pm1 * pm1) if p > 2 else 1 << 40
    for K in {1, 2, 3, 7, min(k64, 512), min(k64, n + 5)}:
        if K * pm1 * pm1 + pm1 < (1 << 64):
            assert oracle.paper_block_dot(p, x, y, K, 64) == want, K
    k32 = ((1 << 32) - pm1 - 1) // (pm1 * pm1) if pm1 * pm1 + pm1 < (1 << 32) else 0
    if k32:
        assert oracle.paper_block_dot(p, x, y, k32, 32) == want
        # one past the Eq. (2) bound is refused
        assert oracle.paper_block_dot(p, x, y, k32 + 1, 32) is None


def test_paper_block_dot_512_threshold():
    """Section 3.4, length-512 blocks in a 32-bit accumulator.  The paper's
    sufficient form 512 p(p-1) < 2^32 stops at 2887 (2897 is the first prime
    over it); the tight Eq. (2) form 512 (p-1)^2 + (p-1) < 2^32 still admits
    2897 and first refuses 2903.  Under the tight form all-(p-1) vectors of
    length 512 must reduce exactly."""
    for p in (2887, 2897):
        x = np.full(512, p - 1, np.uint32)
        assert oracle.paper_block_dot(p, x, x, 512, 32) == 512 % p
    x = np.full(512, 2902, np.uint32)
    assert oracle.paper_block_dot(2903, x, x, 512, 32) is None
    assert 512 * 2887 * 2886 < 2 ** 32 < 512 * 2897 * 2896


@pytest.mark.parametrize("p", [3, 32749, 65521, 2147483647, 4294967291])
def test_paper_overflow_dot_matches(p):
    for n in (0, 1, 5, 4099):
        x = gi.uniform(p, n, 22, 0)
        y = gi.uniform(p, n, 22, 1)
        assert oracle.paper_overflow_dot(p, x, y) == oracle.dot(p, x, y)
    v = np.full(777, p - 1, np.uint32)
    assert oracle.paper_overflow_dot(p, v, v) == 777 % p


def test_paper_fp_reduce_exhaustive_edges():
    for p in (3, 32749, 65521, 67108859, 94906249):
        P = float(p)
        q_max = (1 << 53) // p
        for q in (0, 1, 2, 1000, q_max - 1, q_max):
            for d in (-2, -1, 0, 1, 2, p - 1):
                T = q * p + d
                if 0 <= T <= (1 << 53):
                    assert oracle.paper_fp_reduce(float(T), P) == float(T % p)
        rng = random.Random(p)
        for _ in range(2000):
            T = rng.randrange(0, (1 << 53) + 1)
            assert oracle.paper_fp_reduce(float(T), P) == float(T % p)


@pytest.mark.parametrize("p", [32749, 65521, 67108859])
def test_paper_fp_dot_matches(p):
    n = 2053
    x = gi.uniform(p, n, 23, 0)
    y = gi.uniform(p, n, 23, 1)
    pm1 = p - 1
    kmax = ((1 << 53) - pm1) // (pm1 * pm1)
    for K in {1, 2, kmax}:
        assert oracle.paper_fp_dot(p, x, y, K) == oracle.dot(p, x, y)
    assert oracle.paper_fp_dot(p, x, y, kmax + 1) is None


# ---- GF(p^k): the field arithmetic behind the discrete-logarithm dot product ----

AES_F = [1, 1, 0, 1, 1, 0, 0, 0]   # m(x) = x^8 + x^4 + x^3 + x + 1 (low coefficients)


def _fips_cases():
    here = os.path.dirname(os.path.abspath(__file__))
    for line in open(os.path.join(here, "golden", "fips197_gf256.txt")):
        line = line.split("#")[0].split()
        if line:
            yield line[0], int(line[1], 16), int(line[2], 16), int(line[3], 16)


def test_gfq_fips197_examples():
    cases = list(_fips_cases())
    assert len(cases) == 7
    for op, a, b, want in cases:
        got = oracle.gfq_add(2, 8, a, b) if op == "add" else oracle.gfq_mul(2, 8, AES_F, a, b)
        assert got == want, (op, hex(a), hex(b), hex(got))
    # a dot product of two published products: {57}{83} + {57}{13} = c1 xor fe
    assert oracle.gfq_dot(2, 8, AES_F, [0x57, 0x57], [0x83, 0x13]) == 0xC1 ^ 0xFE


def test_gfq_small_fields_by_hand():
    # GF(4) = GF(2)[x]/(x^2 + x + 1), w = x (value 2): w^2 = w + 1, w (w + 1) = 1, (w + 1)^2 = w
    f4 = [1, 1]
    assert oracle.gfq_mul(2, 2, f4, 2, 2) == 3
    assert oracle.gfq_mul(2, 2, f4, 2, 3) == 1
    assert oracle.gfq_mul(2, 2, f4, 3, 3) == 2
    # GF(9) = GF(3)[x]/(x^2 + 1): x^2 = -1 = 2; (1 + x)^2 = 1 + 2x + x^2 = 2x, value 2*3 = 6
    f9 = [1, 0]
    assert oracle.gfq_mul(3, 2, f9, 3, 3) == 2
    assert oracle.gfq_mul(3, 2, f9, 4, 4) == 6
    # coefficient-wise addition mod p: (2 + 2x) + (1 + 2x) = 0 + x = value 3
    assert oracle.gfq_add(3, 2, 8, 7) == 3


def _field_axioms(p, k, f, triples):
    q = p ** k
    mul = lambda a, b: oracle.gfq_mul(p, k, f, a, b)
    add = lambda a, b: oracle.gfq_add(p, k, a, b)
    for a, b, c in triples:
        assert mul(a, b) == mul(b, a) and add(a, b) == add(b, a)
        assert mul(mul(a, b), c) == mul(a, mul(b, c))
        assert mul(a, add(b, c)) == add(mul(a, b), mul(a, c))
    for a in range(q):
        assert mul(a, 1) == a and add(a, 0) == a and mul(a, 0) == 0
        if a:
            assert any(mul(a, b) == 1 for b in range(1, q)), (p, k, a)


def test_gfq_field_axioms_brute_force():
    import itertools
    for p, k, f in ((2, 3, [1, 1, 0]), (3, 2, [1, 0]), (2, 2, [1, 1])):
        q = p ** k
        _field_axioms(p, k, f, itertools.product(range(q), repeat=3))
    rng = np.random.default_rng(7)
    for p, k in ((5, 2), (3, 3), (7, 2), (2, 8)):
        f = oracle.gfq_find_primitive(p, k)
        _field_axioms(p, k, f, rng.integers(0, p ** k, (300, 3)).tolist())


def test_gfq_frobenius_and_primitive_powers():
    for p, k in ((2, 3), (3, 2), (5, 2), (2, 8), (3, 5)):
        f = oracle.gfq_find_primitive(p, k)
        q = p ** k
        fr = lambda a: oracle.gfq_pow(p, k, f, a, p)
        for a in range(min(q, 60)):
            for b in range(0, min(q, 60), 7):
                assert fr(oracle.gfq_add(p, k, a, b)) == oracle.gfq_add(p, k, fr(a), fr(b))
        # x primitive: its q - 1 powers are the q - 1 distinct non-zero elements
        x = p
        seen, e = set(), 1
        for _ in range(q - 1):
            seen.add(e)
            e = oracle.gfq_mul(p, k, f, e, x)
        assert e == 1 and len(seen) == q - 1 and 0 not in seen


def test_gfq_prime_field_reduces_to_zpz():
    """k = 1: GF(p)[x]/(x + f0) is GF(p) itself; the field dot product equals
    the (separately pinned) Zpz dot product of the residues."""
    for p in (3, 251, 65521, 65537):
        x = gi.uniform(p, 700, 11, 0)
        y = gi.uniform(p, 700, 11, 1)
        f = oracle.gfq_find_primitive(p, 1)
        assert oracle.gfq_dot(p, 1, f, x, y) == oracle.dot(p, x, y)
    # primitivity of x = g in GF(65521) (f = x - g) agrees with Python's modular
    # powers: g is primitive iff g^((p-1)/r) != 1 for each prime r of p - 1
    p = 65521
    for g in range(2, 40):
        py = all(pow(g, (p - 1) // r, p) != 1 for r in (2, 3, 5, 7, 13))
        assert oracle.gfq_x_is_primitive(p, 1, [p - g]) == py, g


def test_gfq_dot_bilinear():
    p, k = 3, 5
    f = oracle.gfq_find_primitive(p, k)
    q = p ** k
    rng = np.random.default_rng(3)
    x, x2, y = (rng.integers(0, q, 200).astype(np.uint32) for _ in range(3))
    s = np.array([oracle.gfq_add(p, k, int(a), int(b)) for a, b in zip(x, x2)], np.uint32)
    assert oracle.gfq_dot(p, k, f, s, y) == oracle.gfq_add(p, k, oracle.gfq_dot(p, k, f, x, y),
                                                          oracle.gfq_dot(p, k, f, x2, y))
    assert oracle.gfq_dot(p, k, f, x[:0], y[:0]) == 0
