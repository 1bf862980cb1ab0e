"""Full-size workloads against the oracle: the 4096-pair batched dot workload
(every result), and the 32768 x 32768 Wiedemann iteration over GF(2^31-1)
(every element of all 64 iterations against the oracle's matrix-vector
product of the previous iterate, plus Freivalds' check per iteration)."""
import numpy as np
import pytest
import torch

import gfp_inputs as gi
import oracle
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def test_batched_workload_full(lib, ctx):
    seed = gi.BASE_SEED + 1
    lens, ps = gi.batched_shapes(4096, seed)
    off, total, x, y = gi.batched_operands(lens, ps, seed)
    want = oracle.dot_batch(ps, lens, off, x, y)
    xd, yd = dev(x), dev(y)
    for repr_, mask in ((0, None), (lib.GFP_REPR_U64_CARRY, None), (lib.GFP_REPR_PERTERM, None),
                        (lib.GFP_REPR_FP64, ps < (1 << 26))):
        sel = np.arange(len(lens)) if mask is None else np.nonzero(mask)[0]
        pairs = [(int(ps[i]), xd[int(off[i]):int(off[i]) + int(lens[i])],
                  yd[int(off[i]):int(off[i]) + int(lens[i])], int(lens[i]), repr_) for i in sel]
        plan = lib.BatchPlan(ctx, pairs)
        out = torch.full((len(sel),), -1, dtype=torch.int32, device="cuda")
        for _ in range(2):
            plan.exec(out)
        torch.cuda.synchronize()
        assert np.array_equal(host(out), want[sel]), repr_
        plan.close()


def test_wiedemann_iteration_full(lib, ctx):
    p, n, iters = 2147483647, 32768, 64
    seed = gi.BASE_SEED + 2
    A = gi.uniform(p, n * n, seed, 0).reshape(n, n)
    x0 = gi.uniform(p, n, seed, 1)
    Ad = dev(A.ravel()).view(n, n)
    Y = torch.full((iters * n,), -1, dtype=torch.int32, device="cuda")
    lib.gfp_matvec_iterate(ctx, p, Ad, dev(x0), Y, iters)
    torch.cuda.synchronize()
    Yh = host(Y).reshape(iters, n)
    del Ad
    # Freivalds per iteration: u^T (A y_{t-1}) = (u^T A) y_{t-1}, w = A^T u from the oracle
    u = gi.uniform(p, n, seed, 2)
    w = oracle.matvec(p, np.ascontiguousarray(A.T), u)
    prev = x0
    for t in range(iters):
        assert oracle.dot(p, u, Yh[t]) == oracle.dot(p, w, prev), t
        # every element: y_t = A y_{t-1}, the oracle's per-term product
        want = oracle.matvec(p, A, prev)
        bad = np.nonzero(Yh[t] != want)[0]
        assert bad.size == 0, (t, bad[:8])
        prev = Yh[t]


@pytest.mark.parametrize("repr_", [0, 1, 3])
def test_dot_beyond_2_31_elements(lib, ctx, repr_):
    """n > 2^31 (64-bit indexing) with all-(p-1) operands at p = 2^32-5:
    every product wraps a 64-bit accumulator; the result is n mod p."""
    p = 4294967291
    n = (1 << 31) + 12345
    ctx.set_repr(repr_)
    try:
        v = torch.full((n,), (p - 1) - (1 << 32), dtype=torch.int32, device="cuda")
        out = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        lib.gfp_dot(ctx, p, v, v, out)
        torch.cuda.synchronize()
        assert int(host(out)[0]) == n % p
    finally:
        ctx.set_repr(0)
        del v
        torch.cuda.empty_cache()


def test_matvec_beyond_2_31_elements(lib, ctx):
    """A with more than 2^31 entries (64-bit row offsets), all (p-1):
    every y_i = cols (p-1)^2 = cols (mod p)."""
    p = 2147483647
    rows, cols = 70001, 32768
    A = torch.full((rows, cols), p - 1, dtype=torch.int32, device="cuda")
    x = torch.full((cols,), p - 1, dtype=torch.int32, device="cuda")
    y = torch.full((rows,), -1, dtype=torch.int32, device="cuda")
    lib.gfp_matvec(ctx, p, A, x, y)
    torch.cuda.synchronize()
    assert (host(y) == cols % p).all()
    del A
    torch.cuda.empty_cache()
