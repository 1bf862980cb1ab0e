"""Service logic without a GPU: the same dispatcher in simulation mode (jobs
complete after a time proportional to their work).  Covers submission,
polling, bounded waits, memory-based admission, queue limits, continuous
batching of dot jobs, cancellation and host-side fault injection."""
import time

import pytest


@pytest.fixture
def srv_factory(lib):
    made = []

    def make(**kw):
        s = lib.Server(simulate=True, **kw)
        made.append(s)
        return s
    yield make
    for s in made:
        s.close()


def test_submit_poll_wait_release(lib, srv_factory):
    s = srv_factory()
    t = s.submit(lib.GFP_JOB_DOT, 65521, n=1 << 16, seed=1)
    st, r = s.wait(t, 2_000_000)
    assert st == lib.GFP_OK and r.status == lib.GFP_OK
    assert r.t_submit_ns <= r.t_admit_ns <= r.t_start_ns <= r.t_done_ns
    st, _ = s.poll(t)
    assert st == lib.GFP_OK
    assert s.release(t) == lib.GFP_OK
    assert s.poll(t)[0] == lib.GFP_ERR_UNKNOWN_TICKET
    assert s.release(t) == lib.GFP_ERR_UNKNOWN_TICKET


def test_matvec_and_block_jobs(lib, srv_factory):
    s = srv_factory()
    h = s.register_matrix(65521, 512, 256, seed=3)
    t1 = s.submit(lib.GFP_JOB_MATVEC, 65521, matrix=h, seed=4)
    t2 = s.submit(lib.GFP_JOB_BLOCK, 65521, matrix=h, nb=64, seed=5)
    for t, elems in ((t1, 512), (t2, 512 * 64)):
        st, r = s.wait(t, 2_000_000)
        assert st == lib.GFP_OK and r.status == lib.GFP_OK and r.out_elems == elems
    # outputs are held until release
    assert s.stats()["mem_in_use"] >= 4 * (512 + 512 * 64)
    s.release(t1)
    s.release(t2)
    assert s.stats()["mem_in_use"] == 0


def test_invalid_jobs_rejected(lib, srv_factory):
    s = srv_factory(mem_budget=1 << 20)
    assert s.submit_status(7, 65521, n=10)[0] == lib.GFP_ERR_INVALID
    assert s.submit_status(lib.GFP_JOB_DOT, 1, n=10)[0] == lib.GFP_ERR_INVALID
    assert s.submit_status(lib.GFP_JOB_MATVEC, 65521, matrix=12345)[0] == lib.GFP_ERR_INVALID
    h = s.register_matrix(65521, 16, 16, seed=1)
    assert s.submit_status(lib.GFP_JOB_MATVEC, 32749, matrix=h)[0] == lib.GFP_ERR_INVALID
    assert s.submit_status(lib.GFP_JOB_BLOCK, 65521, matrix=h, nb=0)[0] == lib.GFP_ERR_INVALID
    # alone larger than the whole budget
    assert s.submit_status(lib.GFP_JOB_DOT, 65521, n=1 << 20)[0] == lib.GFP_ERR_NOMEM


def test_memory_admission_waits_for_space(lib, srv_factory):
    """Each job needs 512 KiB of a 1 MiB budget: at most two at once; every
    job still completes, and the stall counter shows the waits."""
    s = srv_factory(mem_budget=1 << 20)
    ts = [s.submit(lib.GFP_JOB_DOT, 65521, n=1 << 16, seed=i) for i in range(12)]
    for t in ts:
        st, r = s.wait(t, 5_000_000)
        assert st == lib.GFP_OK and r.status == lib.GFP_OK
    stt = s.stats()
    assert stt["completed"] == 12 and stt["mem_peak"] <= 1 << 20
    assert stt["mem_in_use"] == 0


def test_queue_full_is_again(lib, srv_factory):
    s = srv_factory(mem_budget=1 << 20, queue_capacity=4, max_inflight=1)
    h = s.register_matrix(65521, 1 << 14, 1 << 14, seed=1)   # ~1 GiB of simulated work each
    got = [s.submit_status(lib.GFP_JOB_MATVEC, 65521, matrix=h, seed=i)[0] for i in range(12)]
    assert lib.GFP_ERR_AGAIN in got
    assert got[0] == lib.GFP_OK


def test_wait_timeout_then_completion(lib, srv_factory):
    s = srv_factory()
    h = s.register_matrix(65521, 1 << 15, 1 << 15, seed=1)   # 4 GiB: ~0.7 ms simulated
    t = s.submit(lib.GFP_JOB_MATVEC, 65521, matrix=h, seed=2)
    st, _ = s.wait(t, 1)
    assert st in (lib.GFP_ERR_TIMEOUT, lib.GFP_OK)
    st, r = s.wait(t, 5_000_000)
    assert st == lib.GFP_OK and r.status == lib.GFP_OK


def test_dot_jobs_share_launches(lib, srv_factory):
    s = srv_factory(batch_window_us=20000)
    ts = [s.submit(lib.GFP_JOB_DOT, [65521, 4294967291][i % 2], n=1000 + i, seed=i)
          for i in range(200)]
    rs = [s.wait(t, 5_000_000)[1] for t in ts]
    assert all(r.status == lib.GFP_OK for r in rs)
    assert max(r.batch for r in rs) > 1
    assert s.stats()["dot_launches"] < 200


def test_injected_allocation_failures(lib, srv_factory):
    s = srv_factory(fail_every=3)
    ts = [s.submit(lib.GFP_JOB_DOT, 65521, n=4096, seed=i) for i in range(30)]
    rs = [s.wait(t, 5_000_000)[1] for t in ts]
    failed = [r for r in rs if r.status == lib.GFP_ERR_NOMEM]
    ok = [r for r in rs if r.status == lib.GFP_OK]
    assert len(failed) == 10 and len(ok) == 20
    st = s.stats()
    assert st["failed"] == 10 and st["completed"] == 20 and st["mem_in_use"] == 0


def test_release_queued_job_cancels(lib, srv_factory):
    s = srv_factory(max_inflight=1)
    h = s.register_matrix(65521, 1 << 15, 1 << 15, seed=1)
    t1 = s.submit(lib.GFP_JOB_MATVEC, 65521, matrix=h, seed=1)
    t2 = s.submit(lib.GFP_JOB_MATVEC, 65521, matrix=h, seed=2)
    assert s.release(t2) == lib.GFP_OK
    assert s.poll(t2)[0] == lib.GFP_ERR_UNKNOWN_TICKET
    assert s.wait(t1, 5_000_000)[1].status == lib.GFP_OK
    assert s.stats()["cancelled"] == 1


def test_destroy_cancels_pending(lib):
    s = lib.Server(simulate=True, max_inflight=1)
    h = s.register_matrix(65521, 1 << 15, 1 << 15, seed=1)
    for i in range(50):
        s.submit(lib.GFP_JOB_MATVEC, 65521, matrix=h, seed=i)
    t0 = time.time()
    s.close()
    assert time.time() - t0 < 5


def test_memory_budget_from_environment(lib, monkeypatch):
    """mem_budget 0 takes GFP_MEM_BUDGET (bytes) when set."""
    monkeypatch.setenv("GFP_MEM_BUDGET", str(3 << 20))
    s = lib.Server(simulate=True)
    try:
        assert s.stats()["mem_budget"] == 3 << 20
        # a job larger than the budget alone is refused
        st, _ = s.submit_status(lib.GFP_JOB_DOT, 65521, n=1 << 20, seed=1)
        assert st == lib.GFP_ERR_NOMEM
    finally:
        s.close()


def test_prepare_matrix_in_simulation(lib, srv_factory):
    """gfp_prepare_matrix: a no-op in simulation mode for a known matrix,
    GFP_ERR_INVALID for an unknown handle; block jobs still complete."""
    s = srv_factory()
    h = s.register_matrix(65521, 256, 256, seed=9)
    s.prepare_matrix(h)
    s.prepare_matrix(h)   # preparing twice is allowed
    with pytest.raises(lib.GfpError) as ei:
        s.prepare_matrix(h + 1000)
    assert ei.value.status == lib.GFP_ERR_INVALID
    t = s.submit(lib.GFP_JOB_BLOCK, 65521, matrix=h, nb=64, seed=3)
    st, r = s.wait(t, 2_000_000)
    assert st == lib.GFP_OK and r.status == lib.GFP_OK


def test_block_sm_share_and_priority_streams_accepted(lib, srv_factory):
    """The block-SM share and the stream split are accepted in any range; a
    one-stream pool runs every kind on its single stream."""
    for pct, ns in ((0, 1), (50, 2), (100, 3), (150, 8)):
        s = srv_factory(block_sm_percent=pct, n_streams=ns)
        h = s.register_matrix(65521, 128, 128, seed=1)
        ts = [s.submit(lib.GFP_JOB_DOT, 65521, n=1000, seed=2),
              s.submit(lib.GFP_JOB_MATVEC, 65521, matrix=h, seed=3),
              s.submit(lib.GFP_JOB_BLOCK, 65521, matrix=h, nb=64, seed=4)]
        for t in ts:
            st, r = s.wait(t, 2_000_000)
            assert st == lib.GFP_OK and r.status == lib.GFP_OK, (pct, ns)
