"""Parity of the discrete-logarithm (Zech) dot product over GF(p^k) with the
oracle's field arithmetic, through the C ABI: conversions both ways, the dot
product on aligned and unaligned vectors, zero-heavy and cancelling inputs,
field construction errors, and the benchmark's full size."""
import numpy as np
import pytest
import torch

import gfp_inputs as gi
import oracle
from paper_cs_0404008_gb300 import gfpdot as g

pytestmark = pytest.mark.gpu

FIELDS = [(2, 1), (3, 1), (2, 8), (3, 2), (5, 3), (17, 3), (13, 4), (251, 1), (65521, 1),
          (3, 10), (2, 16), (5, 6), (7, 5), (3, 7), (13, 3), (7, 2), (11, 2), (3, 5), (11, 3)]
_F = {}


def field_poly(p, k):
    if (p, k) not in _F:
        _F[(p, k)] = oracle.gfq_find_primitive(p, k)
    return _F[(p, k)]


def dev_u32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


def values(q, n, seed, stream, zeros=0.0):
    v = gi.uniform(q, n, seed, stream) if q > 1 else np.zeros(n, np.uint32)
    if zeros:
        rng = np.random.default_rng(seed + stream)
        v[rng.random(n) < zeros] = 0
    return v


def gpu_dot(fq, xv, yv, offset=0):
    n = xv.shape[0]
    xs = torch.empty(n + offset, dtype=torch.int16, device="cuda")
    ys = torch.empty(n + offset, dtype=torch.int16, device="cuda")
    xc, yc = xs[offset:], ys[offset:]
    fq.to_log(dev_u32(xv), xc, n)
    fq.to_log(dev_u32(yv), yc, n)
    out = torch.full((8,), -1, dtype=torch.int16, device="cuda")
    fq.dot(xc, yc, out, n)
    val = torch.empty(1, dtype=torch.int32, device="cuda")
    fq.from_log(out[:1], val, 1)
    torch.cuda.synchronize()
    assert fq.check() == g.GFP_OK
    assert (out[1:] == -1).all(), "wrote past the output code"
    return int(val.cpu().numpy().view(np.uint32)[0])


@pytest.mark.parametrize("p,k", FIELDS)
def test_dot_matches_oracle(p, k):
    f = field_poly(p, k)
    q = p ** k
    fq = g.Field(p, k, f)
    try:
        for i, (n, zeros, off) in enumerate([(0, 0, 0), (1, 0, 0), (7, 0, 0), (8, 0, 0), (9, 0, 1),
                                             (1000, 0.3, 0), (65541, 0, 3), (1 << 20, 0.01, 0),
                                             ((1 << 20) + 5, 0.5, 1)]):
            xv = values(q, n, 300 + i, 0, zeros)
            yv = values(q, n, 300 + i, 1, zeros)
            assert gpu_dot(fq, xv, yv, off) == oracle.gfq_dot(p, k, f, xv, yv, threads=16), (p, k, n)
    finally:
        fq.close()


@pytest.mark.parametrize("p,k", [(2, 8), (3, 5), (65521, 1), (2, 16)])
def test_conversions_round_trip(p, k):
    f = field_poly(p, k)
    q = p ** k
    fq = g.Field(p, k, f)
    try:
        v = np.arange(q, dtype=np.uint32)
        codes = torch.empty(q, dtype=torch.int16, device="cuda")
        back = torch.empty(q, dtype=torch.int32, device="cuda")
        fq.to_log(dev_u32(v), codes)
        fq.from_log(codes, back)
        torch.cuda.synchronize()
        assert fq.check() == g.GFP_OK
        c = codes.cpu().numpy().view(np.uint16).astype(np.int64)
        assert np.array_equal(back.cpu().numpy().view(np.uint32), v)
        # zero is code 0, 1 is code q-1, the class of x (value p, or -f0 for k = 1) is code 1
        assert c[0] == 0 and c[1] == q - 1
        xval = p if k > 1 else (p - int(f[0])) % p
        assert c[xval] == 1
        # codes are a bijection onto [0, q-1]
        assert sorted(c.tolist()) == list(range(q))
    finally:
        fq.close()


def test_products_and_cancellation():
    """Products through the codes equal the oracle's field products, and a
    sum that cancels gives the zero element."""
    for p, k in ((3, 2), (5, 3), (251, 1), (2, 8)):
        f = field_poly(p, k)
        q = p ** k
        fq = g.Field(p, k, f)
        try:
            rng = np.random.default_rng(5)
            a = rng.integers(0, q, 64).astype(np.uint32)
            b = rng.integers(0, q, 64).astype(np.uint32)
            for i in range(0, 64, 16):
                want = oracle.gfq_mul(p, k, f, int(a[i]), int(b[i]))
                assert gpu_dot(fq, a[i:i + 1], b[i:i + 1]) == want
            # v * 1 + v * (-1) = 0; -1 has constant digit p - 1 (p = 2: -1 = 1)
            minus1 = p - 1
            for v in a[:8]:
                assert gpu_dot(fq, np.array([v, v], np.uint32), np.array([1, minus1], np.uint32)) == 0
            assert gpu_dot(fq, a, np.zeros(64, np.uint32)) == 0
        finally:
            fq.close()


@pytest.mark.parametrize("p,k", [(3, 2), (5, 3), (3, 5), (3, 7), (17, 3), (13, 4), (3, 10), (5, 6), (7, 5)])
def test_accumulator_chains_cancel_and_restart(p, k):
    """Codes 8j+i and 8j+i+4 carry v*1 and v*(-1), so each of a thread's four
    accumulator chains returns to the zero element after every 8-code step
    and restarts from it: the zero-accumulator and cancellation cases of the
    Zech step run in every thread, on the small-field and large-field
    kernels.  One step that does not cancel leaves a nonzero result."""
    f = field_poly(p, k)
    q = p ** k
    fq = g.Field(p, k, f)
    try:
        n = 8 * 40000
        rng = np.random.default_rng(11)
        v = rng.integers(1, q, size=(n // 8, 4)).astype(np.uint32)
        x = np.empty((n // 8, 8), np.uint32)
        y = np.empty((n // 8, 8), np.uint32)
        x[:, :4] = v
        x[:, 4:] = v
        y[:, :4] = 1
        y[:, 4:] = p - 1          # -1: constant digit p - 1
        y[123, 4:] = 1            # this step doubles instead (p > 2)
        x, y = x.reshape(-1), y.reshape(-1)
        want = oracle.gfq_dot(p, k, f, x, y, threads=16)
        assert want != 0
        assert gpu_dot(fq, x, y) == want
        y[123 * 8 + 4:123 * 8 + 8] = p - 1
        assert gpu_dot(fq, x, y) == 0
    finally:
        fq.close()


def test_field_construction_errors():
    with pytest.raises(g.GfpError):
        g.Field(2, 2, [0, 0])          # x^2: not a field
    with pytest.raises(g.GfpError):
        g.Field(3, 2, [1, 0])          # x^2 + 1 is irreducible over GF(3) but x has order 4, not 8
    with pytest.raises(g.GfpError):
        g.Field(4, 1, [1])             # 4 is not prime
    with pytest.raises(g.GfpError):
        g.Field(3, 11, [1] * 11)       # 3^11 > 2^16
    with pytest.raises(g.GfpError):
        g.Field(5, 2, [5, 1])          # coefficient out of range


def test_library_finds_primitive_polynomials():
    for p, k in ((2, 8), (3, 4), (7, 2), (65521, 1), (2, 16)):
        f = g.gfp_gfq_find_primitive(p, k)
        assert oracle.gfq_x_is_primitive(p, k, f), (p, k, f)
    with pytest.raises(g.GfpError):
        g.gfp_gfq_find_primitive(6, 1)


def test_out_of_range_value_is_reported():
    f = field_poly(5, 3)
    fq = g.Field(5, 3, f)
    try:
        codes = torch.empty(4, dtype=torch.int16, device="cuda")
        fq.to_log(dev_u32(np.array([1, 2, 125, 3], np.uint32)), codes)
        assert fq.check() == g.GFP_ERR_RANGE
        assert fq.check() == g.GFP_OK   # cleared
    finally:
        fq.close()


@pytest.mark.parametrize("p,k", [(65521, 1), (2, 8), (3, 10)])
def test_full_size(p, k):
    """The benchmark's size: 2^27 codes per vector (256 MiB each)."""
    f = field_poly(p, k)
    q = p ** k
    n = 1 << 27
    fq = g.Field(p, k, f)
    try:
        xv = values(q, n, 400, 0)
        yv = values(q, n, 400, 1)
        assert gpu_dot(fq, xv, yv) == oracle.gfq_dot(p, k, f, xv, yv, threads=0)
    finally:
        fq.close()
