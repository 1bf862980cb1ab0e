"""The service under the serving workload's own request mix, checked against
the oracle.

The first 2000 requests of the serving workload (the same seeded stream the
benchmark draws: dot products with n up to 2^22, matrix-vector products on
registered matrices up to 16384 x 16384, block products up to 8192 x 8192 x 64,
moduli 65521, 67108859 and 2^32-5) arrive as a Poisson stream at a server
configured as in the benchmark, half of the block matrices prepared (digit
images built at registration) and half not.  Checked against the oracle: every dot
result, every block result whose modulus exceeds 65791 (the residue-pass
path of the tensor-core product), every other block result with p = 65521,
every fourth matrix-vector result and every result on the largest
registered matrix.  A subset is then replayed alone, one job at a time, and
must equal its result in the mix bit for bit (tolerance 0: the results are
exact residues)."""
import threading

import numpy as np
import pytest

import gfp_inputs as gi
import oracle

pytestmark = pytest.mark.gpu

COUNT = 2000
RATE = 20000.0   # jobs per second, about 70 % of the measured capacity of the mix
SEED = gi.BASE_SEED + 5


def test_served_mix_matches_oracle_and_alone(lib):
    import time

    srv = lib.Server(device=0, mem_budget=16 << 30, n_streams=8, batch_window_us=50,
                     max_inflight=256, block_sm_percent=50)
    try:
        specs = gi.serve_pool_specs(SEED)
        handles = {kind: [srv.register_matrix(p, side, side, seed=ms) for p, side, ms in sp]
                   for kind, sp in specs.items()}
        # half of the block matrices carry prepared digit images: block jobs on
        # them take the prepared product, the others convert on every product
        for i in range(0, 16, 2):
            srv.prepare_matrix(handles[2][i])
        reqs = gi.serve_requests(COUNT, SEED)

        def job_p(r):
            return r[1] if r[0] == 0 else specs[r[0]][r[3]][0]

        largest_mv = max(range(16), key=lambda i: specs[1][i][1])
        sample = set()
        for i, r in enumerate(reqs):
            k = r[0]
            if k == 0:
                sample.add(i)
            elif k == 2 and (job_p(r) > 65791 or i % 2 == 0):
                sample.add(i)
            elif k == 1 and (i % 4 == 0 or r[3] == largest_mv):
                sample.add(i)
        assert any(reqs[i][0] == 1 and reqs[i][3] == largest_mv for i in sample)
        assert sum(1 for i in sample if reqs[i][0] == 2 and job_p(reqs[i]) > 65791) > 0

        def submit(r):
            k, p, n, mi, sd = r
            if k == 0:
                return srv.submit(lib.GFP_JOB_DOT, p, n=n, seed=sd)
            mp = specs[k][mi][0]
            if k == 1:
                return srv.submit(lib.GFP_JOB_MATVEC, mp, matrix=handles[1][mi], seed=sd)
            return srv.submit(lib.GFP_JOB_BLOCK, mp, matrix=handles[2][mi], nb=64, seed=sd)

        def collect(i, t):
            st, res = srv.wait(t, 600_000_000)
            assert st == lib.GFP_OK and res.status == lib.GFP_OK, (i, reqs[i], st, res.status)
            if reqs[i][0] == 0:
                out = res.value
            elif i in sample:
                out = srv.result_copy(t, res.out_elems)
            else:
                out = None
            srv.release(t)
            return out, res.batch

        # open-loop Poisson arrivals; a collector waits in submission order
        gaps = -np.log1p(-gi.unit_doubles(SEED, 31, COUNT)) / RATE
        tickets = [None] * COUNT
        results = [None] * COUNT
        ready = threading.Semaphore(0)
        errors = []

        def collector():
            try:
                for i in range(COUNT):
                    ready.acquire()
                    results[i] = collect(i, tickets[i])
            except BaseException as e:   # reported by the main thread
                errors.append(e)

        th = threading.Thread(target=collector, daemon=True)
        th.start()
        t_next = time.perf_counter()
        for i, r in enumerate(reqs):
            t_next += gaps[i]
            while time.perf_counter() < t_next:
                pass
            tickets[i] = submit(r)
            ready.release()
        th.join(900)
        assert not th.is_alive(), "collector did not finish"
        assert not errors, errors[0]
        assert max(b for (_, b), r in zip(results, reqs) if r[0] == 0) > 1, \
            "dot jobs never shared a launch"

        # the oracle, one registered matrix at a time
        by_matrix = {}
        for i in sorted(sample):
            k, p, n, mi, sd = reqs[i]
            if k == 0:
                want = oracle.dot(p, gi.uniform(p, n, sd, 0), gi.uniform(p, n, sd, 1))
                assert results[i][0] == want, (i, reqs[i])
            else:
                by_matrix.setdefault((k, mi), []).append(i)
        for (k, mi), idx in sorted(by_matrix.items()):
            p, side, ms = specs[k][mi]
            A = gi.uniform(p, side * side, ms, 0).reshape(side, side)
            for i in idx:
                sd = reqs[i][4]
                if k == 1:
                    want = oracle.matvec(p, A, gi.uniform(p, side, sd, 0))
                    got = results[i][0]
                else:
                    B = gi.uniform(p, side * 64, sd, 0).reshape(side, 64)
                    want = oracle.block(p, A, B)
                    got = results[i][0].reshape(side, 64)
                bad = np.argwhere(got != want)
                assert bad.size == 0, (i, reqs[i], bad[:4])
            del A

        # a subset alone, one job at a time: identical results
        replay = [i for i in sorted(sample) if reqs[i][0] == 0][:6]
        replay += [i for i in sorted(sample) if reqs[i][0] == 1][:4]
        replay += [i for i in sorted(sample) if reqs[i][0] == 1 and reqs[i][3] == largest_mv][:1]
        replay += [i for i in sorted(sample) if reqs[i][0] == 2 and job_p(reqs[i]) > 65791][:4]
        replay += [i for i in sorted(sample) if reqs[i][0] == 2 and job_p(reqs[i]) == 65521][:2]
        for i in replay:
            out, _ = collect(i, submit(reqs[i]))
            if reqs[i][0] == 0:
                assert out == results[i][0], (i, reqs[i])
            else:
                assert np.array_equal(out, results[i][0]), (i, reqs[i])
    finally:
        srv.close()
