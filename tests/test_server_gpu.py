"""The service on the GPU: every result of a mixed stream of dot, matvec and
block jobs (uneven sizes, three primes, server-generated and caller-owned
operands) equals the oracle, and a sample replayed alone equals its result
in the mix bit for bit (tolerance 0: results are exact residues)."""
import numpy as np
import pytest
import torch

import gfp_inputs as gi
import oracle
from gpu_util import dev, host

pytestmark = pytest.mark.gpu

PR = (65521, 67108859, 4294967291)


@pytest.fixture(scope="module")
def server(lib):
    s = lib.Server(device=0, mem_budget=1 << 30, n_streams=4, batch_window_us=200)
    yield s
    s.close()


def test_mixed_stream_matches_oracle_and_alone(lib, server):
    rng = np.random.default_rng(5)
    mats = []
    for i, (p, r, c) in enumerate(((65521, 700, 1000), (4294967291, 300, 2048),
                                   (67108859, 1024, 640))):
        h = server.register_matrix(p, r, c, seed=900 + i)
        mats.append((h, p, r, c, gi.uniform(p, r * c, 900 + i, 0).reshape(r, c)))
    jobs = []
    for i in range(90):
        kind = rng.choice([0, 0, 0, 1, 2], p=[0.25, 0.25, 0.2, 0.2, 0.1])
        if kind == 0:
            p = int(PR[i % 3])
            n = int(rng.integers(0, 70000))
            jobs.append(("dot", p, n, 5000 + i))
        else:
            h, p, r, c, A = mats[i % 3]
            if kind == 1:
                jobs.append(("mv", p, h, 6000 + i))
            else:
                jobs.append(("blk", p, h, 7000 + i, [64, 17][i % 2]))
    kinds = {"dot": lib.GFP_JOB_DOT, "mv": lib.GFP_JOB_MATVEC, "blk": lib.GFP_JOB_BLOCK}

    def submit(j):
        if j[0] == "dot":
            return server.submit(kinds["dot"], j[1], n=j[2], seed=j[3])
        if j[0] == "mv":
            return server.submit(kinds["mv"], j[1], matrix=j[2], seed=j[3])
        return server.submit(kinds["blk"], j[1], matrix=j[2], nb=j[4], seed=j[3])

    def collect(j, t):
        st, r = server.wait(t, 60_000_000)
        assert st == lib.GFP_OK and r.status == lib.GFP_OK, (j, st, r.status)
        if j[0] == "dot":
            out = r.value
        else:
            out = server.result_copy(t, r.out_elems)
        server.release(t)
        return out, r

    tickets = [submit(j) for j in jobs]
    mixed = [collect(j, t) for j, t in zip(jobs, tickets)]
    matd = {m[0]: m for m in mats}
    for j, (out, r) in zip(jobs, mixed):
        if j[0] == "dot":
            p, n, sd = j[1], j[2], j[3]
            assert out == oracle.dot(p, gi.uniform(p, n, sd, 0), gi.uniform(p, n, sd, 1)), j
        elif j[0] == "mv":
            h, p, rr, c, A = matd[j[2]]
            assert np.array_equal(out, oracle.matvec(p, A, gi.uniform(p, c, j[3], 0))), j
        else:
            h, p, rr, c, A = matd[j[2]]
            B = gi.uniform(p, c * j[4], j[3], 0).reshape(c, j[4])
            assert np.array_equal(out.reshape(rr, j[4]), oracle.block(p, A, B)), j
    assert max(r.batch for _, r in mixed) > 1, "dot jobs never shared a launch"
    # the same jobs alone, one at a time: identical results
    for j, (out, _) in list(zip(jobs, mixed))[::7]:
        out2, r2 = collect(j, submit(j))
        assert r2.batch == 1
        assert np.array_equal(np.asarray(out2), np.asarray(out)), j
    st = server.stats()
    assert st["failed"] == 0 and st["dot_launches"] < sum(1 for j in jobs if j[0] == "dot") + 20


def test_caller_owned_operands(lib, server):
    p, n = 65521, 33333
    x = gi.uniform(p, n, 77, 0)
    y = gi.uniform(p, n, 77, 1)
    xd, yd = dev(x), dev(y)
    t = server.submit(lib.GFP_JOB_DOT, p, n=n, x=xd, y=yd)
    st, r = server.wait(t, 30_000_000)
    assert st == lib.GFP_OK and r.value == oracle.dot(p, x, y)
    server.release(t)
    A = gi.uniform(p, 64 * 80, 78, 0).reshape(64, 80)
    Ad = dev(A.ravel())
    h = server.register_matrix(p, 64, 80, dev=Ad)
    v = gi.uniform(p, 80, 79, 0)
    t = server.submit(lib.GFP_JOB_MATVEC, p, matrix=h, v=dev(v))
    st, r = server.wait(t, 30_000_000)
    assert st == lib.GFP_OK
    assert np.array_equal(server.result_copy(t, 64), oracle.matvec(p, A, v))
    server.release(t)


def test_small_budget_admission_on_gpu(lib):
    s = lib.Server(device=0, mem_budget=1 << 21, n_streams=2)
    try:
        p = 4294967291
        ts = [(s.submit(lib.GFP_JOB_DOT, p, n=1 << 17, seed=i), i) for i in range(16)]
        for t, i in ts:
            st, r = s.wait(t, 30_000_000)
            assert st == lib.GFP_OK and r.status == lib.GFP_OK
            want = oracle.dot(p, gi.uniform(p, 1 << 17, i, 0), gi.uniform(p, 1 << 17, i, 1))
            assert r.value == want
        stt = s.stats()
        assert stt["admission_stalls"] > 0 and stt["mem_peak"] <= 1 << 21
    finally:
        s.close()


def test_large_prime_block_job_on_tensor_cores(lib):
    """A large-p block job big enough for the residue path (five tensor-core
    passes and a recombination, 11 launches): the server pads the matrix rows
    (4099 columns) to 16 bytes so the tensor cores can take it, and the result
    equals the oracle."""
    s = lib.Server(device=0, mem_budget=1 << 30, n_streams=2)
    try:
        p, r, c, nb = 4294967291, 4096, 4099, 64
        h = s.register_matrix(p, r, c, seed=950)
        A = gi.uniform(p, r * c, 950, 0).reshape(r, c)
        before = s.stats()["kernel_launches"]
        t = s.submit(lib.GFP_JOB_BLOCK, p, matrix=h, nb=nb, seed=951)
        st, res = s.wait(t, 60_000_000)
        assert st == lib.GFP_OK and res.status == lib.GFP_OK
        out = s.result_copy(t, res.out_elems).reshape(r, nb)
        s.release(t)
        assert s.stats()["kernel_launches"] - before >= 11
        B = gi.uniform(p, c * nb, 951, 0).reshape(c, nb)
        assert np.array_equal(out, oracle.block(p, A, B))
        # a matvec on the same padded matrix
        t = s.submit(lib.GFP_JOB_MATVEC, p, matrix=h, seed=952)
        st, res = s.wait(t, 60_000_000)
        assert st == lib.GFP_OK and res.status == lib.GFP_OK
        assert np.array_equal(s.result_copy(t, r), oracle.matvec(p, A, gi.uniform(p, c, 952, 0)))
        s.release(t)
    finally:
        s.close()
