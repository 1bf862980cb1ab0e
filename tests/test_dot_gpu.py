"""Parity of the CUDA dot-product, batched and matrix-vector paths with the
oracle, bit for bit, through the C ABI (every result is an exact residue)."""
import numpy as np
import pytest
import torch

import gfp_inputs as gi
import oracle
from gpu_util import dev, dev2, empty, host

pytestmark = pytest.mark.gpu

PRIMES = [2, 3, 7, 251, 32749, 65521, 67108859, 2147483647, 4294967291]
REPRS = [1, 2, 3, 4, 6, 7]   # PERTERM, U64_BLOCK, U64_CARRY, FP64, CENTERED, MONTGOMERY


def eligible(lib, repr_, p):
    prm = lib.gfp_get_params(p)
    if repr_ == lib.GFP_REPR_FP64:
        return bool(prm["fp64_ok"])
    if repr_ == lib.GFP_REPR_MONTGOMERY:
        return prm["k_montgomery"] > 0
    return True


@pytest.fixture
def fresh(ctx):
    ctx.set_repr(0)
    ctx.set_validate(False)
    yield ctx
    ctx.set_repr(0)
    ctx.set_validate(False)


def run_dot(lib, ctx, p, x, y, pad=(0, 0)):
    out = empty(1)
    lib.gfp_dot(ctx, p, dev(x, pad[0]), dev(y, pad[1]), out, n=x.shape[0])
    torch.cuda.synchronize()
    return int(host(out)[0])


@pytest.mark.parametrize("repr_", REPRS)
@pytest.mark.parametrize("p", PRIMES)
def test_dot_parity_sizes(lib, fresh, p, repr_):
    if not eligible(lib, repr_, p):
        pytest.skip("representation not eligible")
    fresh.set_repr(repr_)
    for n in (0, 1, 3, 4, 5, 17, 1000, 4099, 65537, 1 << 20):
        x = gi.uniform(p, n, 100 + n, 0)
        y = gi.uniform(p, n, 100 + n, 1)
        assert run_dot(lib, fresh, p, x, y) == oracle.dot(p, x, y), n


@pytest.mark.parametrize("repr_", REPRS)
def test_dot_unaligned_operands(lib, fresh, repr_):
    for p in (65521, 67108859, 4294967291):
        if not eligible(lib, repr_, p):
            continue
        fresh.set_repr(repr_)
        n = 10007
        x = gi.uniform(p, n, 7, 0)
        y = gi.uniform(p, n, 7, 1)
        for pad in ((1, 0), (0, 3), (2, 2)):
            assert run_dot(lib, fresh, p, x, y, pad) == oracle.dot(p, x, y)


@pytest.mark.parametrize("repr_", REPRS)
@pytest.mark.parametrize("p", [32749, 65521, 67108859, 2147483647, 4294967291])
def test_dot_all_max_stress(lib, fresh, p, repr_):
    """All-(p-1) operands maximise every product: n (p-1)^2 = n (mod p)."""
    if not eligible(lib, repr_, p):
        pytest.skip("representation not eligible")
    fresh.set_repr(repr_)
    for n in (1, 4, 1 << 20, (1 << 22) + 3):
        v = np.full(n, p - 1, np.uint32)
        assert run_dot(lib, fresh, p, v, v) == n % p


def test_dot_auto_matches_and_full_size_workload(lib, fresh):
    """The single-dot workload: p = 65521, n = 2^20, seeded uniform inputs."""
    p, n = 65521, 1 << 20
    x = gi.uniform(p, n, gi.BASE_SEED + 0, 0)
    y = gi.uniform(p, n, gi.BASE_SEED + 0, 1)
    want = oracle.dot(p, x, y)
    assert run_dot(lib, fresh, p, x, y) == want
    # repeated calls reuse the scratch ring (slots return to zero)
    xd, yd, out = dev(x), dev(y), empty(1)
    for _ in range(2000):
        lib.gfp_dot(fresh, p, xd, yd, out)
    torch.cuda.synchronize()
    assert int(host(out)[0]) == want


def random_batch(seed, count, lg_hi=14, primes=gi.PRIMES_BATCHED):
    lens, ps = gi.batched_shapes(count, seed, lg_lo=0.0, lg_hi=lg_hi, primes=primes)
    lens[::17] = 0
    lens[1::13] = 1
    lens[2::11] = 3
    off, total, x, y = gi.batched_operands(lens, ps, seed)
    return lens, ps, off, total, x, y


def batch_pairs(lens, ps, off, xd, yd, repr_=0):
    return [(int(p), xd[int(o):int(o) + int(n)], yd[int(o):int(o) + int(n)], int(n), repr_)
            for n, p, o in zip(lens, ps, off)]


def test_batched_mixed_primes_auto(lib, fresh):
    lens, ps, off, total, x, y = random_batch(11, 700)
    want = oracle.dot_batch(ps, lens, off, x, y)
    xd, yd = dev(x), dev(y)
    out = empty(len(lens))
    lib.gfp_dot_batched(fresh, batch_pairs(lens, ps, off, xd, yd), out)
    torch.cuda.synchronize()
    assert (host(out)[:len(lens)] == want).all()


@pytest.mark.parametrize("repr_", REPRS)
def test_batched_forced_repr(lib, fresh, repr_):
    primes = [p for p in gi.PRIMES_BATCHED if eligible(lib, repr_, p)]
    lens, ps, off, total, x, y = random_batch(12 + repr_, 300, lg_hi=17, primes=primes)
    want = oracle.dot_batch(ps, lens, off, x, y)
    xd, yd = dev(x), dev(y)
    out = empty(len(lens))
    lib.gfp_dot_batched(fresh, batch_pairs(lens, ps, off, xd, yd, repr_), out)
    torch.cuda.synchronize()
    assert (host(out)[:len(lens)] == want).all()


def test_batched_unaligned_pairs(lib, fresh):
    lens, ps, off, total, x, y = random_batch(13, 120)
    want = oracle.dot_batch(ps, lens, off, x, y)
    xd, yd = dev(x, 1), dev(y, 2)   # every pair starts off a 16-byte boundary
    out = empty(len(lens))
    lib.gfp_dot_batched(fresh, batch_pairs(lens, ps, off, xd, yd), out)
    torch.cuda.synchronize()
    assert (host(out)[:len(lens)] == want).all()


def test_batch_plan_reexec_with_new_contents(lib, fresh):
    lens, ps, off, total, x, y = random_batch(14, 400, lg_hi=18)
    xd, yd = dev(x), dev(y)
    plan = lib.BatchPlan(fresh, batch_pairs(lens, ps, off, xd, yd))
    units, nbytes = plan.info()
    assert units >= len(lens) and nbytes == 8 * int(lens.sum())
    out = empty(len(lens))
    for rep in range(3):
        plan.exec(out)
        torch.cuda.synchronize()
        assert (host(out)[:len(lens)] == oracle.dot_batch(ps, lens, off, x, y)).all(), rep
        # new operand contents (same shapes): y <- x
        y = x.copy()
        yd.copy_(xd)
    plan.close()


def test_batched_host_buffers(lib, fresh):
    lens, ps, off, total, x, y = random_batch(15, 500, lg_hi=16)
    want = oracle.dot_batch(ps, lens, off, x, y)
    xh = torch.from_numpy(x.view(np.int32)).pin_memory()
    yh = torch.from_numpy(y.view(np.int32)).pin_memory()
    oh = torch.zeros(len(lens), dtype=torch.int32).pin_memory()
    lib.gfp_dot_batched_host(fresh, ps, lens, off, xh, yh, oh)
    assert (oh.numpy().view(np.uint32) == want).all()
    # a second, smaller call reuses the staging
    lib.gfp_dot_batched_host(fresh, ps[:10], lens[:10], off[:10], xh, yh, oh)
    assert (oh.numpy().view(np.uint32)[:10] == want[:10]).all()


@pytest.mark.parametrize("repr_", [0, 1, 2, 3, 4, 6, 7])
@pytest.mark.parametrize("shape", [(1, 1), (7, 13), (100, 1000), (129, 4097), (300, 32768),
                                   (33, 60000)])
def test_matvec_parity(lib, fresh, shape, repr_):
    m, k = shape
    for p in (65521, 67108859, 2147483647, 4294967291):
        if not eligible(lib, repr_, p):
            continue
        fresh.set_repr(repr_)
        A = gi.uniform(p, m * k, 31, 0).reshape(m, k)
        x = gi.uniform(p, k, 31, 1)
        want = oracle.matvec(p, A, x)
        for ld in (k, k + 1, k + 4):
            y = empty(m)
            lib.gfp_matvec(fresh, p, dev2(A, ld), dev(x), y)
            torch.cuda.synchronize()
            assert (host(y)[:m] == want).all(), (p, ld)


def test_matvec_iterate_graph(lib, fresh):
    """x_{t+1} = A x_t over 8 iterations in one CUDA graph, twice."""
    p, n, iters = 2147483647, 1024, 8
    A = gi.uniform(p, n * n, 41, 0).reshape(n, n)
    x0 = gi.uniform(p, n, 41, 1)
    chain = []
    xt = x0
    for _ in range(iters):
        xt = oracle.matvec(p, A, xt)
        chain.append(xt)
    Ad, xd = dev2(A), dev(x0)
    Y = empty(n * iters)
    for _ in range(2):
        Y.fill_(-1)
        lib.gfp_matvec_iterate(fresh, p, Ad, xd, Y, iters)
        torch.cuda.synchronize()
        got = host(Y)[:n * iters].reshape(iters, n)
        for t in range(iters):
            assert (got[t] == chain[t]).all(), t


def test_fill_uniform_matches_host_generator(lib):
    for p in (2, 65521, 4294967291):
        for off, n in ((0, 1), (0, 1000), (12345, 777)):
            t = empty(n)
            lib.gfp_fill_uniform(p, gi.BASE_SEED, 3, t, n=n, offset=off)
            torch.cuda.synchronize()
            assert (host(t)[:n] == gi.uniform(p, n, gi.BASE_SEED, 3, offset=off)).all()


def test_validation_and_errors(lib, fresh):
    p = 65521
    x = gi.uniform(p, 1000, 5, 0)
    y = x.copy()
    y[500] = p   # not canonical
    out = empty(1)
    fresh.set_validate(True)
    with pytest.raises(lib.GfpError) as ei:
        lib.gfp_dot(fresh, p, dev(x), dev(y), out)
    assert ei.value.status == lib.GFP_ERR_RANGE
    assert run_dot(lib, fresh, p, x, x) == oracle.dot(p, x, x)
    fresh.set_validate(False)
    with pytest.raises(lib.GfpError) as ei:
        lib.gfp_dot(fresh, 1, dev(x), dev(x), out)
    assert ei.value.status == lib.GFP_ERR_INVALID
    fresh.set_repr(lib.GFP_REPR_FP64)
    with pytest.raises(lib.GfpError) as ei:
        lib.gfp_dot(fresh, 2147483647, dev(x), dev(x), out)
    assert ei.value.status == lib.GFP_ERR_UNSUPPORTED
    fresh.set_repr(0)
    # a pointer that is not 4-byte aligned is refused before any launch
    xd = dev(x)
    st = lib.load().gfp_dot(fresh.handle, p, 10, xd.data_ptr() + 2, xd.data_ptr(),
                            out.data_ptr(), None)
    assert st == lib.GFP_ERR_INVALID


@pytest.mark.parametrize("p,n,iters", [(2147483647, 1024, 16), (65521, 777, 5), (4294967291, 1, 3)])
def test_matvec_sequence_projection(lib, fresh, p, n, iters):
    """seq[t] = u^T A^t x0: the fused projection against the oracle chain."""
    A = gi.uniform(p, n * n, 51, 0).reshape(n, n)
    x0 = gi.uniform(p, n, 51, 1)
    u = gi.uniform(p, n, 51, 2)
    want = [oracle.dot(p, u, x0)]
    xt = x0
    for _ in range(iters):
        xt = oracle.matvec(p, A, xt)
        want.append(oracle.dot(p, u, xt))
    Ad, xd, ud = dev2(A), dev(x0), dev(u)
    for use_y in (False, True):
        seq = empty(iters + 1)
        Y = empty(n * iters) if use_y else None
        for _ in range(2):
            seq.fill_(-1)
            lib.gfp_matvec_sequence(fresh, p, Ad, xd, ud, seq, iters, Y=Y)
            torch.cuda.synchronize()
            assert host(seq)[:iters + 1].tolist() == want, use_y
        if use_y:
            assert int(host(Y)[(iters - 1) * n]) == int(xt[0])


@pytest.mark.parametrize("p", [65521, 2147483647])
def test_wiedemann_checkpoint_resume(lib, fresh, p):
    """Checkpoint and resume of the iteration: 64 steps in one call equal 32
    steps, the state (t = 32, x_32) saved to the host and the device copies
    dropped, then 32 more steps started from the restored x_32.  The scalar
    sequence u^T A^t x resumes the same way: the second half's sequence is
    the tail of the whole one.  Both are checked against the oracle chain."""
    n, iters, half = 1536, 64, 32
    A = gi.uniform(p, n * n, 53, 0).reshape(n, n)
    x0 = gi.uniform(p, n, 53, 1)
    u = gi.uniform(p, n, 53, 2)
    Ad, ud = dev2(A), dev(u)
    Y = empty(n * iters)
    lib.gfp_matvec_iterate(fresh, p, Ad, dev(x0), Y, iters)
    seq = empty(iters + 1)
    lib.gfp_matvec_sequence(fresh, p, Ad, dev(x0), ud, seq, iters)
    torch.cuda.synchronize()
    whole, whole_seq = host(Y)[:n * iters].reshape(iters, n), host(seq)[:iters + 1]
    # first half, then a checkpoint on the host
    Y1 = empty(n * half)
    lib.gfp_matvec_iterate(fresh, p, Ad, dev(x0), Y1, half)
    torch.cuda.synchronize()
    ckpt = {"t": half, "x": host(Y1)[(half - 1) * n:half * n].copy()}
    del Y1
    torch.cuda.empty_cache()
    # resume from the checkpoint
    Y2 = empty(n * half)
    lib.gfp_matvec_iterate(fresh, p, Ad, dev(ckpt["x"]), Y2, iters - ckpt["t"])
    seq2 = empty(iters - half + 1)
    lib.gfp_matvec_sequence(fresh, p, Ad, dev(ckpt["x"]), ud, seq2, iters - half)
    torch.cuda.synchronize()
    assert np.array_equal(host(Y2)[:n * half].reshape(half, n), whole[half:])
    assert np.array_equal(host(seq2)[:iters - half + 1], whole_seq[half:])
    # the oracle chain, every element of every step
    xt = x0
    for t in range(iters):
        assert int(oracle.dot(p, u, xt)) == int(whole_seq[t]), t
        xt = oracle.matvec(p, A, xt)
        assert np.array_equal(whole[t], xt), t
    assert int(oracle.dot(p, u, xt)) == int(whole_seq[iters])
