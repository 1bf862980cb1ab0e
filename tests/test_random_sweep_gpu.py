"""Seeded random sweep of the CUDA paths against the oracle: moduli at the
edges of every bound (the Zpz and Eq. (2) thresholds, the fp16 digit range
of the tensor cores, the FP64 eligibility limit, a delay bound of 16),
ragged shapes, unaligned starts, every eligible representation, uniform and
all-(p-1) operands; tensor-core block products also with A prepared once.
Each case is compared bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import dev, dev2, empty, host

pytestmark = pytest.mark.gpu

PRIMES = [2, 3, 5, 13, 251, 257, 2887, 2897, 2903, 32749, 46337, 65521, 65537, 65789, 65809,
          94906249, 94906297, 1073741789, 3037000493, 2147483647, 4294967291]
CUDA_CORE_REPRS = [0, 1, 2, 3, 4, 6, 7]   # AUTO, PERTERM, U64_BLOCK, U64_CARRY, FP64, CENTERED, MONTGOMERY


def eligible(lib, r, p):
    prm = lib.gfp_get_params(p)
    if r == lib.GFP_REPR_FP64:
        return bool(prm["fp64_ok"])
    if r == lib.GFP_REPR_MONTGOMERY:
        return prm["k_montgomery"] > 0
    return True


def operands(rng, p, shape, maxed):
    if maxed:
        return np.full(shape, p - 1, dtype=np.uint32)
    return rng.integers(0, p, size=shape, dtype=np.uint64).astype(np.uint32)


@pytest.fixture
def fresh(ctx):
    ctx.set_repr(0)
    ctx.set_validate(False)
    yield ctx
    ctx.set_repr(0)


@pytest.mark.parametrize("seed", range(24))
def test_random_dots_and_matvecs(lib, fresh, seed):
    rng = np.random.default_rng(1000 + seed)
    for case in range(12):
        p = int(rng.choice(PRIMES))
        r = int(rng.choice([x for x in CUDA_CORE_REPRS if eligible(lib, x, p)]))
        fresh.set_repr(r)
        maxed = case % 4 == 0
        n = int(rng.integers(0, 70000))
        x, y = operands(rng, p, n, maxed), operands(rng, p, n, maxed)
        pad = (int(rng.integers(0, 4)), int(rng.integers(0, 4)))
        out = empty(1)
        lib.gfp_dot(fresh, p, dev(x, pad[0]), dev(y, pad[1]), out, n=n)
        torch.cuda.synchronize()
        assert int(host(out)[0]) == oracle.dot(p, x, y), (seed, case, p, r, n, pad)
        rows, cols = int(rng.integers(1, 300)), int(rng.integers(1, 900))
        A = operands(rng, p, (rows, cols), maxed)
        xv = operands(rng, p, cols, maxed)
        ld = cols + int(rng.integers(0, 5))
        yv = empty(rows)
        lib.gfp_matvec(fresh, p, dev2(A, ld), dev(xv), yv)
        torch.cuda.synchronize()
        assert np.array_equal(host(yv)[:rows], oracle.matvec(p, A, xv)), (seed, case, p, r, rows, cols, ld)


@pytest.mark.parametrize("seed", range(24))
def test_random_block_products(lib, fresh, seed):
    rng = np.random.default_rng(2000 + seed)
    for case in range(8):
        p = int(rng.choice(PRIMES))
        tc = case % 2 == 0          # tensor cores (directly or through residues) or CUDA cores
        if tc:
            fresh.set_repr(lib.GFP_REPR_F16TC)
        else:
            fresh.set_repr(int(rng.choice([x for x in CUDA_CORE_REPRS if eligible(lib, x, p)])))
        m, k, nb = int(rng.integers(1, 300)), int(rng.integers(1, 2100)), int(rng.integers(1, 140))
        maxed = case % 4 == 1
        A, B = operands(rng, p, (m, k), maxed), operands(rng, p, (k, nb), maxed)
        lda = (k + 3) // 4 * 4 + 4 * int(rng.integers(0, 2))   # 16-byte rows for the TMA path
        ldb = nb + int(rng.integers(0, 3))
        ldc = nb + int(rng.integers(0, 3))
        Cfull = torch.full((m, ldc), -1, dtype=torch.int32, device="cuda")
        lib.gfp_matmul_block(fresh, p, dev2(A, lda), dev2(B, ldb), Cfull[:, :nb])
        torch.cuda.synchronize()
        assert lib.gfp_context_check(fresh) == lib.GFP_OK
        out = host(Cfull)
        assert (out[:, nb:] == 0xFFFFFFFF).all(), "wrote outside C"
        want = oracle.block(p, A, B)
        assert np.array_equal(out[:, :nb], want), (seed, case, p, tc, m, k, nb)
        if tc:
            # the same product with A prepared once (any row stride), C rewritten
            prep = lib.BlockPrep(fresh, p, dev2(A, k + int(rng.integers(0, 3))))
            try:
                Cfull.fill_(-1)
                prep.matmul(fresh, dev2(B, ldb), Cfull[:, :nb])
                torch.cuda.synchronize()
                assert lib.gfp_context_check(fresh) == lib.GFP_OK
                out = host(Cfull)
                assert (out[:, nb:] == 0xFFFFFFFF).all(), "wrote outside C"
                assert np.array_equal(out[:, :nb], want), ("prepared", seed, case, p, m, k, nb)
            finally:
                prep.close()


@pytest.mark.parametrize("seed", range(16))
def test_random_sparse_row_products(lib, fresh, seed):
    rng = np.random.default_rng(3000 + seed)
    for case in range(6):
        p = int(rng.choice(PRIMES))
        fresh.set_repr(int(rng.choice([x for x in CUDA_CORE_REPRS if eligible(lib, x, p)])))
        m, k, nb = int(rng.integers(1, 200)), int(rng.integers(1, 3000)), 4 * int(rng.integers(1, 40))
        dens = float(rng.choice([0.0, 0.01, 0.1, 0.5]))
        maxed = case % 3 == 0
        cols, vals, row_ptr = [], [], [0]
        for _ in range(m):
            c = np.nonzero(rng.random(k) < dens)[0].astype(np.uint32)
            cols.append(c)
            vals.append(operands(rng, p, c.shape[0], maxed))
            row_ptr.append(row_ptr[-1] + c.shape[0])
        col = np.concatenate(cols) if cols else np.zeros(0, np.uint32)
        val = np.concatenate(vals) if vals else np.zeros(0, np.uint32)
        row_ptr = np.array(row_ptr, dtype=np.uint32)
        B = operands(rng, p, (k, nb), maxed)
        one = np.zeros(1, np.uint32)
        C = torch.full((m, nb), -1, dtype=torch.int32, device="cuda")
        lib.gfp_matmul_block_csr(fresh, p, k, dev(row_ptr), dev(col) if col.size else dev(one),
                                 dev(val) if val.size else dev(one), dev2(B), C)
        torch.cuda.synchronize()
        assert np.array_equal(host(C), oracle.csr(p, row_ptr, col, val, B)), (seed, case, p, m, k, nb, dens)
