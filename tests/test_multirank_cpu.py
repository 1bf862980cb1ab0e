"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): each
rank works on its own batch (weak scaling, no data-path collective) and the
step time is the maximum over ranks.  The per-rank work is the oracle on a
small batch, so no GPU is involved."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import time

    import torch.distributed as dist

    import bench
    import gfp_inputs as gi
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seed = bench.rank_seed(rank)
    lens, ps = gi.batched_shapes(64, seed, lg_lo=4.0, lg_hi=10.0)
    off, total, x, y = gi.batched_operands(lens, ps, seed)
    dist.barrier()
    t0 = time.perf_counter()
    res = oracle.dot_batch(ps, lens, off, x, y, threads=1)
    dt = time.perf_counter() - t0 + 0.01 * rank     # rank 1 is made slower
    tmax = bench.reduce_max(dt)
    out[rank] = (seed, float(lens.sum()), dt, tmax, int(res.sum()))
    dist.destroy_process_group()


def test_two_rank_weak_scaling_and_max_time():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    r0, r1 = out[0], out[1]
    assert r0[0] != r1[0], "ranks must draw different batches"
    assert r0[3] == r1[3] == max(r0[2], r1[2]), "step time is the max over ranks"
    assert r0[1] > 0 and r1[1] > 0
