"""gfp_dot_batched_noalloc: the batched dot product for callers that cannot
allocate device memory (fixed scratch array inside the library).

Collected last on purpose.  Its results must equal those of gfp_dot_batched,
the allocating entry point, bit for bit (exact residues, tolerance 0), on two
calls in a row; it must also refuse batches beyond its fixed limits."""
import numpy as np
import pytest
import torch

import gfp_inputs as gi
from gpu_util import dev, empty, host

pytestmark = pytest.mark.gpu


def make_batch(seed, count, lg_hi):
    lens, ps = gi.batched_shapes(count, seed, lg_lo=0.0, lg_hi=lg_hi)
    lens[::9] = 0
    lens[1::7] = 5
    off, total, x, y = gi.batched_operands(lens, ps, seed)
    xd, yd = dev(x), dev(y)
    pairs = [(int(p), xd[int(o):int(o) + int(n)], yd[int(o):int(o) + int(n)], int(n))
             for n, p, o in zip(lens, ps, off)]
    return pairs


def test_noalloc_matches_batched_two_calls(lib, ctx):
    ctx.set_repr(0)
    for call, (seed, count, lg_hi) in enumerate(((501, 1024, 18.0), (502, 333, 20.0))):
        pairs = make_batch(seed, count, lg_hi)
        want = empty(count)
        lib.gfp_dot_batched(ctx, pairs, want)
        got = empty(count)
        lib.gfp_dot_batched_noalloc(pairs, got)
        torch.cuda.synchronize()
        assert np.array_equal(host(got)[:count], host(want)[:count]), call


def test_noalloc_repeated_same_inputs(lib, ctx):
    pairs = make_batch(503, 200, 16.0)
    want = empty(200)
    lib.gfp_dot_batched(ctx, pairs, want)
    for _ in range(2):
        got = empty(200)
        lib.gfp_dot_batched_noalloc(pairs, got)
        torch.cuda.synchronize()
        assert np.array_equal(host(got)[:200], host(want)[:200])


def test_noalloc_rejects_beyond_limits(lib):
    x = torch.zeros(8, dtype=torch.int32, device="cuda")
    out = empty(1025)
    with pytest.raises(lib.GfpError) as ei:
        lib.gfp_dot_batched_noalloc([(65521, x, x, 8)] * 1025, out)
    assert ei.value.status == lib.GFP_ERR_INVALID
    # one pair whose length needs more than 16384 work units of 65536 elements
    big = (1 << 30) + 1
    with pytest.raises(lib.GfpError) as ei:
        lib.gfp_dot_batched_noalloc([(65521, x.data_ptr(), x.data_ptr(), big)], out)
    assert ei.value.status == lib.GFP_ERR_INVALID
