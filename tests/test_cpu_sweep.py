"""The host representations of the paper's dot-product comparison (Section 3,
Figures 5-8): every variant gives the oracle's residue wherever it claims its
domain, its block length is the largest one its bound allows, and the domain
edges follow the paper's word-size limits."""
import numpy as np
import pytest

import gfp_inputs as gi
import oracle
from paper_cs_0404008_gb300 import sweep

PRIMES = [2, 3, 5, 7, 251, 2887, 2897, 2903, 32749, 40009, 40499, 46337, 65521, 65537,
          92681, 1048573, 94906249, 94906267, 2147483647, 3037000493, 4294967291]
LENGTHS = [0, 1, 7, 511, 512, 513, 3000]


@pytest.mark.parametrize("v", sweep.VARIANTS)
def test_variant_matches_oracle(v):
    checked = 0
    for p in PRIMES:
        if not sweep.supported(v, p):
            continue
        for i, n in enumerate(LENGTHS):
            x = gi.uniform(p, n, 90 + i, 0)
            y = gi.uniform(p, n, 90 + i, 1)
            assert sweep.dot(v, p, x, y) == oracle.dot(p, x, y), (v, p, n)
        # every entry p - 1: the largest products, so every accumulator wraps or
        # reaches its block bound
        m = np.full(3000, p - 1, np.uint32)
        assert sweep.dot(v, p, m, m) == oracle.dot(p, m, m), (v, p, "max")
        # centred extremes: (p-1)/2 and (p+1)/2 are the largest magnitudes of both signs
        h = np.array([(p - 1) // 2, (p + 1) // 2 % p] * 700, np.uint32)
        assert sweep.dot(v, p, h, h[::-1].copy()) == oracle.dot(p, h, h[::-1].copy()), (v, p, "half")
        checked += 1
    assert checked >= 3, v


@pytest.mark.parametrize("v", sweep.VARIANTS)
def test_time_returns_the_same_residue(v):
    p = 32749 if sweep.supported(v, 32749) else 65521
    x, y = gi.uniform(p, 512, 91, 0), gi.uniform(p, 512, 91, 1)
    sec, r = sweep.time(v, p, x, y, 50)
    assert sec > 0 and r == oracle.dot(p, x, y)


def test_domains_follow_the_word_size_limits():
    # Section 2.1: unsigned 32-bit AXPY r + ab <= p(p-1) < 2^32 up to 65521 (and 65536)
    assert sweep.supported("zpz32", 65521) and sweep.supported("zpz32", 65536)
    assert not sweep.supported("zpz32", 65537)
    assert sweep.supported("overflow32", 65521) and not sweep.supported("overflow32", 65537)
    # 64-bit words take every p < 2^32
    for v in ("zpz64", "block64", "overflow64", "hybrid64"):
        assert sweep.supported(v, 4294967291) and sweep.supported(v, 2)
    # Montgomery needs an odd modulus below its B
    for v in ("montgomery_block16", "montgomery_block32"):
        assert not sweep.supported(v, 2) and not sweep.supported(v, 65536)
    assert sweep.supported("montgomery_block16", 65521)
    assert not sweep.supported("montgomery_block16", 65537)
    assert sweep.supported("montgomery_block32", 4294967291)
    # doubles: one exact product plus the carried residue below 2^53
    for p in (94906249, 94906265, 94906267):
        assert sweep.supported("fp53_block", p) == (p * (p - 1) <= 2 ** 53)
    assert not sweep.supported("fp53_block", 2147483647)


@pytest.mark.parametrize("v,limit,carried", [
    ("block32", 2 ** 32 - 1, True), ("hybrid32", 2 ** 32 - 1, True),
    ("block64", 2 ** 64 - 1, True), ("hybrid64", 2 ** 64 - 1, True),
    ("fp53_block", 2 ** 53, True)])
def test_block_lengths_are_maximal(v, limit, carried):
    for p in (3, 251, 2897, 32749, 65521, 1048573, 94906249, 2147483647, 4294967291):
        lam = sweep.block(v, p)
        if lam == 0:
            assert (p - 1) ** 2 + (p - 1) > limit
            continue
        assert lam * (p - 1) ** 2 + (p - 1) <= limit
        assert (lam + 1) * (p - 1) ** 2 + (p - 1) > limit


def test_block_lengths_of_the_other_bounds():
    for p in (3, 251, 2897, 32749, 65521):
        h = p // 2
        lam = sweep.block("centered_block32", p)
        assert lam * h * h + (p - 1) <= 2 ** 31 - 1 < (lam + 1) * h * h + (p - 1)
        lam = sweep.block("montgomery_block16", p)
        assert lam * (p - 1) ** 2 < p * 2 ** 16 <= (lam + 1) * (p - 1) ** 2
    for p in (3, 65521, 2147483647, 4294967291):
        lam = sweep.block("montgomery_block32", p)
        assert lam * (p - 1) ** 2 < p * 2 ** 32 <= (lam + 1) * (p - 1) ** 2


def test_the_512_threshold_of_section_3_4():
    """On 512-long vectors the 32-bit block and hybrid variants need one final
    reduction only while a block covers all 512 terms: up to 2897 with the
    tight bound lambda (p-1)^2 + (p-1) < 2^32 (2887 is the last prime of the
    sufficient form 512 p(p-1) < 2^32; 2903 is the first refused)."""
    assert sweep.block("hybrid32", 2887) >= 512
    assert sweep.block("hybrid32", 2897) >= 512
    assert sweep.block("hybrid32", 2903) < 512


def test_errors():
    x = np.zeros(4, np.uint32)
    with pytest.raises(ValueError):
        sweep.dot("zpz32", 65537, x, x)
    with pytest.raises(ValueError):
        sweep.dot("montgomery_block32", 10, x, x)
    assert sweep.name(0) == "zpz32" and sweep.name(99) is None
    assert sweep.block(0, 1) == 0
