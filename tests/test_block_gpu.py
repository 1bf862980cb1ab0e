"""Parity of the block products (tensor-core and CUDA-core dense paths, and
the sparse-row path) with the oracle, bit for bit, through the C ABI."""
import numpy as np
import pytest
import torch

import gfp_inputs as gi
import oracle
from gpu_util import dev, dev2, host

pytestmark = pytest.mark.gpu


@pytest.fixture
def fresh(ctx):
    ctx.set_repr(0)
    ctx.set_validate(False)
    yield ctx
    ctx.set_repr(0)
    ctx.set_validate(False)
    assert ctx is not None


def run_block(lib, ctx, p, A, B, lda=None, ldb=None, ldc=None):
    m, k = A.shape
    nb = B.shape[1]
    Ad, Bd = dev2(A, lda), dev2(B, ldb)
    Cfull = torch.full((m, ldc or nb), -1, dtype=torch.int32, device="cuda")
    Cd = Cfull[:, :nb]
    lib.gfp_matmul_block(ctx, p, Ad, Bd, Cd)
    torch.cuda.synchronize()
    assert lib.gfp_context_check(ctx) == lib.GFP_OK
    out = host(Cfull)
    if ldc and ldc > nb:
        assert (out[:, nb:] == 0xFFFFFFFF).all(), "wrote outside C"
    return out[:, :nb]


def run_prepared(lib, ctx, p, A, Bs, lda=None, ldc=None):
    """Prepare A once, then one product per B in Bs; returns the C matrices."""
    m, k = A.shape
    prep = lib.BlockPrep(ctx, p, dev2(A, lda))
    outs = []
    try:
        for B in Bs:
            nb = B.shape[1]
            Cfull = torch.full((m, ldc or nb), -1, dtype=torch.int32, device="cuda")
            prep.matmul(ctx, dev2(B), Cfull[:, :nb])
            torch.cuda.synchronize()
            assert lib.gfp_context_check(ctx) == lib.GFP_OK
            out = host(Cfull)
            if ldc and ldc > nb:
                assert (out[:, nb:] == 0xFFFFFFFF).all(), "wrote outside C"
            outs.append(out[:, :nb])
    finally:
        prep.close()
    return outs


SHAPES_TC = [(1, 1, 1), (7, 13, 5), (128, 64, 64), (129, 1000, 64), (300, 2049, 70),
             (64, 4101, 3), (257, 1025, 128), (130, 3000, 65)]


@pytest.mark.parametrize("shape", SHAPES_TC)
@pytest.mark.parametrize("p", [2, 3, 251, 32749, 65521, 65537, 65789])
def test_block_tensor_core_parity(lib, fresh, p, shape):
    fresh.set_repr(lib.GFP_REPR_F16TC)
    m, k, nb = shape
    A = gi.uniform(p, m * k, 61, 0).reshape(m, k)
    B = gi.uniform(p, k * nb, 61, 1).reshape(k, nb)
    lda = (k + 3) // 4 * 4   # the tensor-core path streams A rows with 16-byte loads
    got = run_block(lib, fresh, p, A, B, lda=lda)
    assert np.array_equal(got, oracle.block(p, A, B)), (p, shape)
    # a row stride that is not a multiple of 4 cannot take the tensor-core path
    if lda == k and k % 4 == 0:
        with pytest.raises(lib.GfpError) as ei:
            run_block(lib, fresh, p, A, B, lda=k + 1)
        assert ei.value.status == lib.GFP_ERR_UNSUPPORTED


def test_block_tensor_core_strides(lib, fresh):
    fresh.set_repr(lib.GFP_REPR_F16TC)
    p, m, k, nb = 65521, 200, 1500, 64
    A = gi.uniform(p, m * k, 62, 0).reshape(m, k)
    B = gi.uniform(p, k * nb, 62, 1).reshape(k, nb)
    want = oracle.block(p, A, B)
    for lda, ldb, ldc in ((k + 4, nb, nb), (k + 12, nb + 3, nb + 5)):
        assert np.array_equal(run_block(lib, fresh, p, A, B, lda, ldb, ldc), want)


@pytest.mark.parametrize("p", [65521, 65537, 65789])
def test_block_tensor_core_extreme_digits(lib, fresh, p):
    """Residues whose centred value is +-(p-1)/2 give digits of magnitude 128:
    every 1024-term chunk of digit products reaches 2^24 exactly."""
    fresh.set_repr(lib.GFP_REPR_F16TC)
    h = (p - 1) // 2
    m, k, nb = 256, 4096, 64
    rng = np.random.default_rng(p)
    A = np.where(rng.random((m, k)) < 0.5, h, p - h).astype(np.uint32)
    B = np.where(rng.random((k, nb)) < 0.5, h, p - h).astype(np.uint32)
    A[:, :1024] = h
    B[:1024, :] = h
    got = run_block(lib, fresh, p, A, B)
    assert np.array_equal(got, oracle.block(p, A, B))
    # all-equal case against the closed form k * h^2 mod p
    A1 = np.full((128, 2048), h, np.uint32)
    B1 = np.full((2048, 64), h, np.uint32)
    assert (run_block(lib, fresh, p, A1, B1) == (2048 * h * h) % p).all()


def test_block_auto_path_and_unsupported(lib, fresh):
    p = 65521
    A = gi.uniform(p, 50 * 70, 63, 0).reshape(50, 70)
    B = gi.uniform(p, 70 * 9, 63, 1).reshape(70, 9)
    assert np.array_equal(run_block(lib, fresh, p, A, B), oracle.block(p, A, B))
    fresh.set_repr(lib.GFP_REPR_F16TC)
    # the tensor cores need A 16-byte aligned with lda a multiple of 4 (k = 70 here)
    with pytest.raises(lib.GfpError) as ei:
        run_block(lib, fresh, 2147483647, A, B)
    assert ei.value.status == lib.GFP_ERR_UNSUPPORTED


@pytest.mark.parametrize("repr_", [0, 1, 2, 3, 4, 6, 7])
@pytest.mark.parametrize("p", [65521, 67108859, 2147483647, 4294967291])
def test_block_cuda_core_parity(lib, fresh, p, repr_):
    if repr_ == lib.GFP_REPR_FP64 and not lib.gfp_get_params(p)["fp64_ok"]:
        pytest.skip("not eligible")
    fresh.set_repr(repr_)
    for m, k, nb in ((1, 1, 1), (65, 33, 64), (100, 700, 70), (3, 2000, 129)):
        A = gi.uniform(p, m * k, 64, 0).reshape(m, k)
        B = gi.uniform(p, k * nb, 64, 1).reshape(k, nb)
        assert np.array_equal(run_block(lib, fresh, p, A, B, k + 1, nb + 2, nb + 1),
                              oracle.block(p, A, B)), (m, k, nb)


def test_block_k_zero_writes_zeros(lib, fresh):
    A = torch.zeros((5, 4), dtype=torch.int32, device="cuda")[:, :0]
    B = torch.zeros((0, 7), dtype=torch.int32, device="cuda")
    C = torch.full((5, 7), -1, dtype=torch.int32, device="cuda")
    lib.gfp_matmul_block(fresh, 65521, A, B, C)
    torch.cuda.synchronize()
    assert (host(C) == 0).all()


RNS_PRIMES = [65797, 1000003, 67108859, 2147483647, 4294967291]
RNS_SHAPES = [(1, 1, 1), (7, 13, 5), (129, 1000, 64), (300, 2049, 70), (64, 4101, 3), (257, 1025, 128)]


def _pad4(k):
    return (k + 3) // 4 * 4


@pytest.mark.parametrize("p", RNS_PRIMES)
def test_block_rns_tensor_core_parity(lib, fresh, p):
    """p above the direct digit range: residues modulo several primes <= 65791
    on the tensor cores, recombined modulo p (forced and automatic path)."""
    for i, (m, k, nb) in enumerate(RNS_SHAPES):
        A = gi.uniform(p, m * k, 66 + i, 0).reshape(m, k)
        B = gi.uniform(p, k * nb, 66 + i, 1).reshape(k, nb)
        want = oracle.block(p, A, B)
        fresh.set_repr(lib.GFP_REPR_F16TC)
        assert np.array_equal(run_block(lib, fresh, p, A, B, lda=_pad4(k)), want), (p, m, k, nb)
        fresh.set_repr(lib.GFP_REPR_AUTO)
        assert np.array_equal(run_block(lib, fresh, p, A, B, lda=_pad4(k), ldc=nb + 3), want)


@pytest.mark.parametrize("p", [67108859, 4294967291])
def test_block_rns_largest_sums(lib, fresh, p):
    """Every entry p - 1: each exact sum is k (p-1)^2, the bound the moduli
    must cover; the result is the closed form k mod p."""
    fresh.set_repr(lib.GFP_REPR_F16TC)
    for m, k, nb in ((128, 4096, 64), (200, 20000, 64)):
        A = np.full((m, k), p - 1, np.uint32)
        B = np.full((k, nb), p - 1, np.uint32)
        assert (run_block(lib, fresh, p, A, B) == k % p).all(), (p, k)


def test_block_rns_matches_cuda_core_path(lib, fresh):
    p, m, k, nb = 2147483647, 384, 3000, 64
    A = gi.uniform(p, m * k, 67, 0).reshape(m, k)
    B = gi.uniform(p, k * nb, 67, 1).reshape(k, nb)
    fresh.set_repr(lib.GFP_REPR_F16TC)
    tc = run_block(lib, fresh, p, A, B, lda=_pad4(k))
    fresh.set_repr(lib.GFP_REPR_U64_CARRY)
    cc = run_block(lib, fresh, p, A, B, lda=_pad4(k))
    assert np.array_equal(tc, cc)
    assert np.array_equal(tc, oracle.block(p, A, B))


def test_block_rns_full_size(lib, fresh):
    """16384 x 16384 x 64 over GF(2^32 - 5) on the tensor cores (five residue
    passes), every entry against the oracle."""
    p, m, k, nb = 4294967291, 16384, 16384, 64
    seed = gi.BASE_SEED + 8
    A = gi.uniform(p, m * k, seed, 0).reshape(m, k)
    B = gi.uniform(p, k * nb, seed, 1).reshape(k, nb)
    got = run_block(lib, fresh, p, A, B)
    want = oracle.block(p, A, B)
    assert np.array_equal(got, want)
    assert np.array_equal(run_prepared(lib, fresh, p, A, [B])[0], want)


def test_block_many_units_per_cta(lib, fresh):
    """4096 x 16384 x 64: 32 row tiles x 32 exact chunks, several (tile,
    chunk) units per persistent CTA, so shared-memory slots, TMEM stages and
    accumulator sets are reused many times within one launch."""
    p, m, k, nb = 65521, 4096, 16384, 64
    A = gi.uniform(p, m * k, 65, 0).reshape(m, k)
    B = gi.uniform(p, k * nb, 65, 1).reshape(k, nb)
    for _ in range(2):
        assert np.array_equal(run_block(lib, fresh, p, A, B), oracle.block(p, A, B))


def test_block_long_k_residue_sums_stay_below_2_32(lib):
    """One output over K = 2^26 + 2^16 terms: 65600 exact 1024-term chunks,
    each built to leave the residue p - 1 (A all ones, B the constant c with
    1024 c = p - 1 mod p), so that the chunk residues of the output sum to
    65600 (p - 1) > 2^32.  The tensor-core kernel keeps every running sum of
    residues below p; a plain 32-bit sum of them would wrap.  Needs a 16 GiB
    B digit image (one 16 KiB tile per 64-deep k-block), held by a context of
    its own and freed with it."""
    p = 65521
    k = (1 << 26) + (1 << 16)
    c = (p - 1) * pow(1024, -1, p) % p
    A = np.ones((1, k), dtype=np.uint32)
    B = np.full((k, 1), c, dtype=np.uint32)
    want = oracle.block(p, A, B)
    assert int(want[0, 0]) == (k // 1024) * (p - 1) % p   # the chunks as built
    ctx = lib.Context(0)
    try:
        ctx.set_repr(lib.GFP_REPR_F16TC)
        got = run_block(lib, ctx, p, A, B)
        assert np.array_equal(got, want), (got, want)
    finally:
        ctx.close()


def test_block_full_size_workload(lib, fresh):
    """The block workload: A 16384 x 16384, B 16384 x 64 over GF(65521),
    tensor-core path, every entry against the oracle."""
    p, m, k, nb = 65521, 16384, 16384, 64
    seed = gi.BASE_SEED + 3
    A = gi.uniform(p, m * k, seed, 0).reshape(m, k)
    B = gi.uniform(p, k * nb, seed, 1).reshape(k, nb)
    got = run_block(lib, fresh, p, A, B)
    want = oracle.block(p, A, B)
    assert np.array_equal(got, want)
    assert np.array_equal(run_prepared(lib, fresh, p, A, [B])[0], want)


@pytest.mark.parametrize("repr_", [0, 1, 2, 3, 6, 7])
def test_csr_parity(lib, fresh, repr_):
    fresh.set_repr(repr_)
    for p in (65521, 4294967291):
        for m, k, nb, dens in ((1, 1, 1, 1.0), (50, 300, 64, 0.01), (200, 500, 70, 0.2),
                               (33, 64, 130, 0.5)):
            row_ptr, col, val = gi.csr_pattern(m, k, dens, p, seed=71)
            B = gi.uniform(p, k * nb, 71, 9999).reshape(k, nb)
            C = torch.full((m, nb), -1, dtype=torch.int32, device="cuda")
            lib.gfp_matmul_block_csr(fresh, p, k, dev(row_ptr), dev(col) if col.size else dev(np.zeros(1, np.uint32)),
                                     dev(val) if val.size else dev(np.zeros(1, np.uint32)), dev2(B), C)
            torch.cuda.synchronize()
            assert np.array_equal(host(C), oracle.csr(p, row_ptr, col, val, B)), (p, m, k, nb)


def _csr_run(lib, ctx, p, k, row_ptr, col, val, B, ldb=None, ldc=None, Bd=None):
    m, nb = row_ptr.shape[0] - 1, B.shape[1]
    one = np.zeros(1, np.uint32)
    Cfull = torch.full((m, ldc or nb), -1, dtype=torch.int32, device="cuda")
    C = Cfull[:, :nb]
    lib.gfp_matmul_block_csr(ctx, p, k, dev(row_ptr), dev(col) if col.size else dev(one),
                             dev(val) if val.size else dev(one), dev2(B, ldb) if Bd is None else Bd, C)
    torch.cuda.synchronize()
    return host(C)


@pytest.mark.parametrize("repr_", [0, 2, 3])
def test_csr_wide_shapes(lib, fresh, repr_):
    """The 16-byte-gather sparse-row kernel (nb and ldb multiples of 4): several
    64-column groups with a ragged last group, rows spanning many 32-nonzero
    chunks with ragged tails, empty rows, padded leading dimensions and a C
    whose rows are not 16-byte aligned."""
    fresh.set_repr(repr_)
    for p in (65521, 4294967291):
        for m, k, nb, dens, ldb, ldc in ((300, 5000, 128, 0.05, None, None),
                                         (40, 3000, 132, 0.3, 136, 133),
                                         (64, 100, 4, 1.0, 8, 5),
                                         (257, 700, 64, 0.0, None, None),
                                         (100, 2000, 192, 0.02, 196, None)):
            row_ptr, col, val = gi.csr_pattern(m, k, dens, p, seed=73)
            B = gi.uniform(p, k * nb, 73, 5).reshape(k, nb)
            got = _csr_run(lib, fresh, p, k, row_ptr, col, val, B, ldb, ldc)
            assert np.array_equal(got, oracle.csr(p, row_ptr, col, val, B)), (p, m, k, nb, ldb, ldc)


def test_csr_unaligned_b_takes_the_general_kernel(lib, fresh):
    """B rows not 16-byte aligned (a view one element into its storage) and
    an odd leading dimension: the general sparse-row kernel, same results."""
    p, m, k, nb = 65521, 80, 900, 64
    row_ptr, col, val = gi.csr_pattern(m, k, 0.1, p, seed=74)
    B = gi.uniform(p, k * nb, 74, 1).reshape(k, nb)
    want = oracle.csr(p, row_ptr, col, val, B)
    store = torch.zeros(k * nb + 1, dtype=torch.int32, device="cuda")
    store[1:].copy_(torch.from_numpy(B.reshape(-1).view(np.int32)))
    Bd = store[1:].view(k, nb)
    assert Bd.data_ptr() % 16 != 0
    assert np.array_equal(_csr_run(lib, fresh, p, k, row_ptr, col, val, B, Bd=Bd), want)
    assert np.array_equal(_csr_run(lib, fresh, p, k, row_ptr, col, val, B, ldb=nb + 1), want)


@pytest.mark.parametrize("p,lam", [(554000009, 60), (1073741789, 16), (1073741827, 15)])
def test_csr_rows_around_the_delay_bound(lib, fresh, p, lam):
    """Blocked representation at moduli with delay bounds of 60, 16 and 15
    products, rows of 90-130 nonzeros at the largest residues.  The wide
    kernel adds plain 64-bit sums and reduces them after every floor(lambda/16)
    chunks of 32 nonzeros (three chunks; every chunk, where a half adds exactly
    lambda products; below 16 the representation's own accumulators): an
    accumulator that overflowed would change the residue."""
    fresh.set_repr(lib.GFP_REPR_U64_BLOCK)
    k, nb = 400, 64
    assert lib.gfp_delay_bound(p, 64, 1) == lam
    rng = np.random.default_rng(75)
    rows_c, rows_v = [], []
    for length in range(90, 131):
        rows_c.append(np.sort(rng.choice(k, size=length, replace=False)).astype(np.uint32))
        v = np.full(length, p - 1, np.uint32) if length % 2 == 0 else \
            rng.integers(0, p, size=length, dtype=np.uint64).astype(np.uint32)
        rows_v.append(v)
    row_ptr = np.concatenate([[0], np.cumsum([len(c) for c in rows_c])]).astype(np.uint32)
    col, val = np.concatenate(rows_c), np.concatenate(rows_v)
    B = np.full((k, nb), p - 1, np.uint32)
    B[:, nb // 2:] = rng.integers(0, p, size=(k, nb - nb // 2), dtype=np.uint64).astype(np.uint32)
    got = _csr_run(lib, fresh, p, k, row_ptr, col, val, B)
    assert np.array_equal(got, oracle.csr(p, row_ptr, col, val, B))


def test_csr_k_zero_writes_zeros(lib, fresh):
    p, m, nb = 65521, 5, 8
    row_ptr = np.zeros(m + 1, np.uint32)
    C = torch.full((m, nb), -1, dtype=torch.int32, device="cuda")
    one = dev(np.zeros(1, np.uint32))
    B = torch.zeros((0, nb), dtype=torch.int32, device="cuda")
    lib.gfp_matmul_block_csr(fresh, p, 0, dev(row_ptr), one, one, B, C)
    torch.cuda.synchronize()
    assert np.array_equal(host(C), np.zeros((m, nb), np.uint32))


def test_csr_full_size_workload(lib, fresh):
    """The sparse-row workload: CSR A 16384 x 16384 at density 0.01 times B
    16384 x 64 over GF(65521), every entry against the oracle."""
    p, m, k, nb = 65521, 16384, 16384, 64
    seed = gi.BASE_SEED + 3
    row_ptr, col, val = gi.csr_pattern(m, k, 0.01, p, seed)
    B = gi.uniform(p, k * nb, seed, 1).reshape(k, nb)
    got = _csr_run(lib, fresh, p, k, row_ptr, col, val, B)
    assert np.array_equal(got, oracle.csr(p, row_ptr, col, val, B))


def test_csr_validation(lib, fresh):
    p, m, k, nb = 65521, 10, 20, 8
    row_ptr, col, val = gi.csr_pattern(m, k, 0.3, p, seed=72)
    B = gi.uniform(p, k * nb, 72, 1).reshape(k, nb)
    C = torch.zeros((m, nb), dtype=torch.int32, device="cuda")
    fresh.set_validate(True)
    bad = col.copy()
    bad[0] = k   # column out of range
    with pytest.raises(lib.GfpError) as ei:
        lib.gfp_matmul_block_csr(fresh, p, k, dev(row_ptr), dev(bad), dev(val), dev2(B), C)
    assert ei.value.status == lib.GFP_ERR_INVALID
    lib.gfp_matmul_block_csr(fresh, p, k, dev(row_ptr), dev(col), dev(val), dev2(B), C)
    torch.cuda.synchronize()
    assert np.array_equal(host(C), oracle.csr(p, row_ptr, col, val, B))


def test_bounded_wait_expires_and_context_survives(lib, fresh):
    """A pipeline wait that nothing satisfies gives up after its limit and
    reports GFP_ERR_TIMEOUT; the context keeps working afterwards."""
    import time
    t0 = time.time()
    assert lib.gfp_wait_selftest(50_000_000) == lib.GFP_ERR_TIMEOUT
    assert time.time() - t0 < 5
    assert lib.gfp_wait_selftest(10) == lib.GFP_ERR_INVALID
    p = 65521
    A = gi.uniform(p, 128 * 256, 80, 0).reshape(128, 256)
    B = gi.uniform(p, 256 * 64, 80, 1).reshape(256, 64)
    fresh.set_repr(lib.GFP_REPR_F16TC)
    assert np.array_equal(run_block(lib, fresh, p, A, B), oracle.block(p, A, B))


@pytest.mark.parametrize("shape", SHAPES_TC)
@pytest.mark.parametrize("p", [2, 251, 65521, 65789, 2147483647, 4294967291])
def test_block_prepared_parity(lib, fresh, p, shape):
    """A prepared once (8-bit digit planes, one image per residue modulus for
    p > 65536),
    then two products with different B: both equal the oracle and the
    unprepared product.  Ragged row tiles, ragged k-blocks and exact chunks,
    ragged column tiles; any row stride of A (the preparation reads A with
    plain loads)."""
    m, k, nb = shape
    A = gi.uniform(p, m * k, 62, 0).reshape(m, k)
    B1 = gi.uniform(p, k * nb, 62, 1).reshape(k, nb)
    B2 = gi.uniform(p, k * nb, 62, 2).reshape(k, nb)
    got = run_prepared(lib, fresh, p, A, [B1, B2], lda=k + 1, ldc=nb + 3)
    assert np.array_equal(got[0], oracle.block(p, A, B1)), (p, shape)
    assert np.array_equal(got[1], oracle.block(p, A, B2)), (p, shape)


@pytest.mark.parametrize("p", [257, 65521, 65536, 65789, 4294967291])
def test_block_prepared_extreme_digits(lib, fresh, p):
    """A's entries at both ends of its representatives (t = min((p-1)/2,
    32639) kept as itself, t + 1 taken as t + 1 - p: digits 127 and -128),
    B's at the ends of the centred range, and all (p-1), over 5000 terms
    (five exact chunks)."""
    m, k, nb = 256, 5000, 64
    h = (p - 1) // 2
    t = min(h, 32639)
    for a_val, b_val in ((t, h), (t + 1, h + 1), (t, h + 1), (t + 1, h), (p - 1, p - 1)):
        A = np.full((m, k), a_val, np.uint32)
        B = np.full((k, nb), b_val, np.uint32)
        want = oracle.block(p, A[:1], B)
        got = run_prepared(lib, fresh, p, A, [B])[0]
        assert (got == want[0][None, :]).all(), (p, a_val, b_val)


def test_block_prepared_info_and_errors(lib, fresh):
    m, k = 300, 1000
    A = dev2(gi.uniform(65521, m * k, 63, 0).reshape(m, k))
    prep = lib.BlockPrep(fresh, 65521, A)
    kb, mt = (k + 63) // 64, (m + 127) // 128
    assert prep.info() == (mt * kb * 16384, 1)   # two 8-bit planes per 128 x 64 tile
    B = dev2(gi.uniform(65521, (k + 1) * 8, 63, 1).reshape(k + 1, 8))
    C = torch.zeros((m, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        prep.matmul(fresh, B, C)   # k mismatch is refused before the call
    prep.close()
    prep = lib.BlockPrep(fresh, 4294967291, A)
    assert prep.info()[1] >= 2
    prep.close()
    with pytest.raises(lib.GfpError) as ei:
        lib.BlockPrep(fresh, 1, A)
    assert ei.value.status == lib.GFP_ERR_INVALID
