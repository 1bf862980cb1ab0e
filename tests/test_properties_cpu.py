"""Randomised properties (hypothesis) on the host side: the library's host
reductions and bounds against Python integers, the host sweep variants
against the oracle, and the field laws of the oracle's GF(p^k) arithmetic.
No GPU needed; skipped where hypothesis is not installed."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import gfp_inputs as gi  # noqa: E402
import oracle  # noqa: E402
from paper_cs_0404008_gb300 import sweep  # noqa: E402

PRIMES = [2, 3, 5, 7, 251, 2887, 2897, 32749, 40009, 65521, 65537, 1048573, 67108859,
          94906249, 2147483647, 3037000493, 4294967291]
moduli = st.one_of(st.sampled_from(PRIMES), st.integers(2, 2 ** 32 - 1))
SET = settings(max_examples=150, deadline=None)


@SET
@given(p=moduli, x=st.integers(0, 2 ** 64 - 1))
def test_reduce_u64_is_the_remainder(lib, p, x):
    assert lib.gfp_reduce_u64(x, p) == x % p


@SET
@given(p=st.integers(2, 94906265), t=st.integers(0, 2 ** 53))
def test_reduce_f64_is_the_remainder(lib, p, t):
    assert lib.gfp_reduce_f64(float(t), p) == float(t % p)


@SET
@given(p=moduli, bits=st.sampled_from([32, 53, 64]), carried=st.booleans())
def test_delay_bound_is_the_largest_safe_block(lib, p, bits, carried):
    k = lib.gfp_delay_bound(p, bits, int(carried))
    q = (p - 1) ** 2
    extra = (p - 1) if carried else 0
    lim = 2 ** bits - 1          # strict: lambda (p-1)^2 (+ (p-1)) < 2^m
    if q == 0:
        return
    if k == 0:
        assert q + extra > lim
    else:
        assert k * q + extra <= lim and (k + 1) * q + extra > lim


@SET
@given(v=st.sampled_from(sweep.VARIANTS), p=st.sampled_from(PRIMES), n=st.integers(0, 1500),
       seed=st.integers(0, 2 ** 32 - 1), maxed=st.booleans())
def test_sweep_variant_equals_oracle(v, p, n, seed, maxed):
    if not sweep.supported(v, p):
        return
    if maxed:
        x = np.full(n, p - 1, np.uint32)
        y = gi.uniform(p, n, seed, 1)
    else:
        x, y = gi.uniform(p, n, seed, 0), gi.uniform(p, n, seed, 1)
    assert sweep.dot(v, p, x, y) == oracle.dot(p, x, y)


FIELDS = [(2, 3), (2, 8), (3, 2), (3, 5), (5, 3), (7, 2), (13, 2), (251, 1)]
_F = {}


def _poly(p, k):
    if (p, k) not in _F:
        _F[(p, k)] = oracle.gfq_find_primitive(p, k)
    return _F[(p, k)]


@SET
@given(fk=st.sampled_from(FIELDS), data=st.data())
def test_gfq_field_laws(fk, data):
    p, k = fk
    q = p ** k
    f = _poly(p, k)
    a, b, c = (data.draw(st.integers(0, q - 1)) for _ in range(3))
    mul = lambda u, v: oracle.gfq_mul(p, k, f, u, v)
    add = lambda u, v: oracle.gfq_add(p, k, u, v)
    assert mul(a, add(b, c)) == add(mul(a, b), mul(a, c))
    assert mul(mul(a, b), c) == mul(a, mul(b, c))
    assert mul(a, b) == mul(b, a)
    # a^(q-1) = 1 for a != 0 (Lagrange), a^q = a for all a
    assert oracle.gfq_pow(p, k, f, a, q) == a
    if a:
        assert oracle.gfq_pow(p, k, f, a, q - 1) == 1


@SET
@given(fk=st.sampled_from(FIELDS), n=st.integers(0, 300), seed=st.integers(0, 2 ** 32 - 1))
def test_gfq_dot_is_bilinear_and_splits(fk, n, seed):
    p, k = fk
    q = p ** k
    f = _poly(p, k)
    x, y = gi.uniform(q, n, seed, 0), gi.uniform(q, n, seed, 1)
    h = n // 2
    whole = oracle.gfq_dot(p, k, f, x, y)
    assert whole == oracle.gfq_add(p, k, oracle.gfq_dot(p, k, f, x[:h], y[:h]),
                                   oracle.gfq_dot(p, k, f, x[h:], y[h:]))
    assert whole == oracle.gfq_dot(p, k, f, x, y, threads=4)
