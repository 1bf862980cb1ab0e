"""gfp_dot_batched_noalloc: the batched dot product for callers that cannot
allocate device memory (fixed scratch array inside the library).

Collected last on purpose, so that a run stopping at the first failure has
already run every other test.  Its results must equal the oracle's residues
element by element (exact, tolerance 0) and those of gfp_dot_batched, the
allocating entry point, on two calls in a row; it must also refuse batches
beyond its fixed limits without enqueuing anything."""
import numpy as np
import pytest
import torch

import gfp_inputs as gi
import oracle
from gpu_util import dev, empty, host

pytestmark = pytest.mark.gpu


def make_batch(seed, count, lg_hi):
    lens, ps = gi.batched_shapes(count, seed, lg_lo=0.0, lg_hi=lg_hi)
    lens[::9] = 0
    lens[1::7] = 5
    off, total, x, y = gi.batched_operands(lens, ps, seed)
    want = oracle.dot_batch(ps, lens, off, x, y)
    xd, yd = dev(x), dev(y)
    pairs = [(int(p), xd[int(o):int(o) + int(n)], yd[int(o):int(o) + int(n)], int(n))
             for n, p, o in zip(lens, ps, off)]
    return pairs, want


def test_noalloc_matches_oracle_two_calls(lib, ctx):
    ctx.set_repr(0)
    for call, (seed, count, lg_hi) in enumerate(((501, 1024, 18.0), (502, 333, 20.0))):
        pairs, want = make_batch(seed, count, lg_hi)
        got = empty(count)
        lib.gfp_dot_batched_noalloc(pairs, got)
        ref = empty(count)
        lib.gfp_dot_batched(ctx, pairs, ref)
        torch.cuda.synchronize()
        assert np.array_equal(host(got)[:count], want), call
        assert np.array_equal(host(got)[:count], host(ref)[:count]), call


def test_noalloc_repeated_same_inputs(lib):
    pairs, want = make_batch(503, 200, 16.0)
    for _ in range(2):
        got = empty(200)
        lib.gfp_dot_batched_noalloc(pairs, got)
        torch.cuda.synchronize()
        assert np.array_equal(host(got)[:200], want)


def _k_of(lib, p, r):
    pr = lib.gfp_get_params(p)
    return {lib.GFP_REPR_U64_BLOCK: pr["k_u64"], lib.GFP_REPR_FP64: pr["k_fp64"],
            lib.GFP_REPR_CENTERED: pr["k_centered"],
            lib.GFP_REPR_MONTGOMERY: pr["k_montgomery"]}.get(r, 0)


@pytest.mark.parametrize("p", [67108859, 2147483647, 4294967291])
def test_noalloc_each_representation_near_its_bound(lib, ctx, p):
    """Every representation named explicitly, on all-(p-1) and uniform operands
    whose lengths sit around the representation's block length k."""
    reprs = [lib.GFP_REPR_PERTERM, lib.GFP_REPR_U64_BLOCK, lib.GFP_REPR_U64_CARRY,
             lib.GFP_REPR_FP64, lib.GFP_REPR_CENTERED, lib.GFP_REPR_MONTGOMERY]
    pr = lib.gfp_get_params(p)
    descs, ps, lens, xs, ys = [], [], [], [], []
    off = 0
    for r in reprs:
        if r == lib.GFP_REPR_FP64 and not pr["fp64_ok"]:
            continue
        if r == lib.GFP_REPR_MONTGOMERY and p % 2 == 0:
            continue
        k = _k_of(lib, p, r) or 64
        for n in sorted({1, max(1, k - 1), k, k + 1, 2 * k + 1, 70001}):
            for kind in ("max", "uniform"):
                if kind == "max":
                    xv = np.full(n, p - 1, dtype=np.uint32)
                    yv = xv.copy()
                else:
                    xv = gi.uniform(p, n, 900 + r, 2 * len(lens))
                    yv = gi.uniform(p, n, 900 + r, 2 * len(lens) + 1)
                pad = (-n) % 4
                descs.append((r, off, n))
                ps.append(p)
                lens.append(n)
                xs.append(np.concatenate([xv, np.zeros(pad, np.uint32)]))
                ys.append(np.concatenate([yv, np.zeros(pad, np.uint32)]))
                off += n + pad
    x, y = np.concatenate(xs), np.concatenate(ys)
    offs = np.array([o for _, o, _ in descs], dtype=np.int64)
    want = oracle.dot_batch(np.array(ps), np.array(lens), offs, x, y)
    xd, yd = dev(x), dev(y)
    pairs = [(p, xd[o:o + n], yd[o:o + n], n, r) for r, o, n in descs]
    count = len(pairs)
    for _ in range(2):
        got = empty(count)
        lib.gfp_dot_batched_noalloc(pairs, got)
        ref = empty(count)
        lib.gfp_dot_batched(ctx, pairs, ref)
        torch.cuda.synchronize()
        assert np.array_equal(host(got)[:count], want)
        assert np.array_equal(host(got)[:count], host(ref)[:count])


def test_noalloc_refuses_tensor_core_representation(lib):
    x = torch.zeros(8, dtype=torch.int32, device="cuda")
    out = empty(1)
    with pytest.raises(lib.GfpError) as ei:
        lib.gfp_dot_batched_noalloc([(65521, x, x, 8, lib.GFP_REPR_F16TC)], out)
    assert ei.value.status == lib.GFP_ERR_UNSUPPORTED


def test_noalloc_rejects_beyond_limits(lib):
    """Each over-limit batch also carries a descriptor that is refused with a
    different status (a forced tensor-core representation, which no dot
    product takes), and every descriptor is checked before anything is
    written or enqueued: if the limit check under test were broken, the call
    would return that other status instead of launching."""
    x = torch.zeros(8, dtype=torch.int32, device="cuda")
    out = empty(1025)
    tc = (65521, x, x, 8, lib.GFP_REPR_F16TC)
    ok = (65521, x, x, 8)
    with pytest.raises(lib.GfpError) as ei:
        lib.gfp_dot_batched_noalloc([tc] + [ok] * 1024, out)
    assert ei.value.status == lib.GFP_ERR_INVALID
    # one pair whose length needs more than 16384 work units of 65536 elements
    big = (65521, x.data_ptr(), x.data_ptr(), (1 << 30) + 1)
    with pytest.raises(lib.GfpError) as ei:
        lib.gfp_dot_batched_noalloc([big, tc], out)
    assert ei.value.status == lib.GFP_ERR_INVALID
    # the scratch still serves a valid call afterwards
    pairs, want = make_batch(504, 64, 12.0)
    got = empty(64)
    lib.gfp_dot_batched_noalloc(pairs, got)
    torch.cuda.synchronize()
    assert np.array_equal(host(got)[:64], want)
