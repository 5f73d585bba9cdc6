"""The job server's scheduling on the host (vp_server_create_fake: the same
admission, pool accounting and reporting as the GPU server, jobs running on
a host clock for C microseconds). No GPU: these cover first-come admission
by idle lane and pool space, head-of-line waiting, the pool's bookkeeping,
the drain deadline, reporting each job once, the trace replay
(vp_server_replay) and the age-priority ranks (vp_server_set_policy).
"""
import time

import pytest

import paper_2602_12098_gb300 as vp

K, M, N_PATHS = 16, 16, 256


def per_channel_bytes():
    # the state layout of one channel (the library rounds each piece to 256 B)
    return 24 * K * K + 16 * K * M + 20 * N_PATHS + 5 * K + 300


def job(C, S=14):
    # pointers are never dereferenced by the fake executor; they must be non-null
    return vp.job_desc(K, M, 256, N_PATHS, C, S, 16, 16, 16, 16, 16)


def drain_all(srv, timeout=20.0):
    srv.drain(timeout)
    return srv.poll()


def test_jobs_complete_and_are_reported_once():
    with vp.Server(1 << 30, lanes=3, fake=True) as srv:        # host bookkeeping only
        ids = [srv.submit(job(C)) for C in (2000, 3000, 1000, 500, 4000, 800)]
        done = drain_all(srv)
        assert sorted(r[0] for r in done) == sorted(ids)
        assert all(r[1] == 0 and 0.0 <= r[2] <= r[3] for r in done)
        assert srv.poll() == []
        st = srv.stats()
        assert st["completed"] == st["submitted"] == 6 and st["queued"] == 0 and st["in_flight"] == 0
        assert st["pool_used"] == 0 and 1 < st["max_in_flight"] <= 3


def test_simulated_run_time_and_lanes():
    """Each job holds a lane for C microseconds: four 20 ms jobs on two lanes
    take two rounds."""
    with vp.Server(4 << 30, lanes=2, fake=True) as srv:      # host bookkeeping only: nothing allocated
        srv.reset_clock()
        for _ in range(4):
            srv.submit(job(20000))
        done = sorted(drain_all(srv), key=lambda r: r[0])
        for r in done:
            assert r[3] - r[2] == pytest.approx(20.0, abs=0.5)
        # the third and fourth start when the first two end
        assert done[2][2] >= done[0][3] - 0.5 and done[3][2] >= done[1][3] - 0.5
        assert srv.stats()["max_in_flight"] == 2


def test_admission_waits_for_pool_space_first_come():
    """A job that does not fit waits at the head of the queue and the jobs
    behind it wait too (first come, first served), until space frees up."""
    unit = per_channel_bytes()
    pool = 10000 * unit + (1 << 20)
    with vp.Server(pool, lanes=4, fake=True) as srv:
        srv.reset_clock()
        a = srv.submit(job(6000))       # 6 ms, 6000 channels of state
        b = srv.submit(job(7000))       # does not fit beside a: waits
        c = srv.submit(job(100))        # would fit, but queues behind b
        st = srv.stats()
        assert st["in_flight"] == 1 and st["queued"] == 2
        done = {r[0]: r for r in drain_all(srv)}
        assert done[b][2] >= done[a][3] - 0.2          # b admitted after a ended
        assert done[c][2] >= done[b][2] - 0.2          # c not before b
        assert srv.stats()["pool_high_water"] <= pool


def test_pool_accounting_coalesces():
    unit = per_channel_bytes()
    with vp.Server(8000 * unit + (1 << 20), lanes=8, fake=True) as srv:
        for _ in range(4):
            srv.submit(job(2000))                   # 2 ms each: all four still running below
        st = srv.stats()
        assert st["in_flight"] == 4 and st["pool_used"] >= 4 * 2000 * unit
        drain_all(srv)
        # freed pieces merge back: a job of nearly the whole pool fits again
        srv.submit(job(8000))
        assert srv.stats()["in_flight"] == 1
        drain_all(srv)
        assert srv.stats()["pool_used"] == 0


def test_drain_deadline_and_refusals():
    with vp.Server(1 << 30, lanes=1, fake=True) as srv:
        with pytest.raises(vp.VPError) as e:         # larger than the whole pool
            srv.submit(job(100000))
        assert e.value.code == 6
        with pytest.raises(vp.VPError) as e:         # out-of-range descriptor
            srv.submit(vp.job_desc(17, 16, 256, 256, 10, 14, 16, 16, 16, 16, 16))
        assert e.value.code == 1
        srv.submit(job(30000))                      # 30 ms
        t0 = time.perf_counter()
        with pytest.raises(vp.VPError) as e:
            srv.drain(0.005)
        assert e.value.code == 4 and time.perf_counter() - t0 < 1.0
        drain_all(srv)
        assert srv.stats()["completed"] == 1


def test_destroy_with_waiting_jobs():
    srv = vp.Server(2 << 20, lanes=1, fake=True)
    for _ in range(3):
        srv.submit(job(10))
    srv.close()


def test_replay_submits_at_arrival_times():
    """vp_server_replay submits each job when the host clock reaches its
    arrival time, reports every job of the trace in trace order, and leaves
    nothing for vp_server_poll."""
    arrivals = [0.0, 0.5, 0.5, 3.0, 3.2, 8.0]          # ms
    sizes = [1000, 2000, 500, 300, 4000, 700]          # us of fake run time
    with vp.Server(1 << 30, lanes=2, fake=True) as srv:
        recs, sub = srv.replay([job(C) for C in sizes], arrivals, timeout_s=20.0)
        assert [r[0] for r in recs] == sorted(r[0] for r in recs)
        for a, s, r, C in zip(arrivals, sub, recs, sizes):
            assert r[1] == 0
            assert s >= a and s - a < 50.0            # dispatch lag of the replay loop (ms, loose for CI)
            assert r[2] >= s - 1e-3                     # admitted no earlier than submitted
            assert r[3] - r[2] == pytest.approx(C * 1e-3, abs=0.5)
        # two lanes: the third job (arriving with the second) waits for the first to end
        assert recs[2][2] >= recs[0][3] - 0.2
        assert srv.poll() == []
        st = srv.stats()
        assert st["completed"] == st["submitted"] == len(sizes) and st["in_flight"] == 0


def test_replay_refusals_leave_server_untouched():
    with vp.Server(1 << 30, lanes=2, fake=True) as srv:
        for arr in ([1.0, 0.5], [-1.0, 0.0], [0.0, float("nan")]):   # decreasing, negative, NaN
            with pytest.raises(vp.VPError) as e:
                srv.replay([job(10), job(10)], arr)
            assert e.value.code == 1
        with pytest.raises(vp.VPError) as e:                          # one job larger than the pool
            srv.replay([job(10), job(100000)], [0.0, 0.0])
        assert e.value.code == 6
        assert srv.stats()["submitted"] == 0
        srv.submit(job(20000))                                        # busy server: refused
        with pytest.raises(vp.VPError) as e:
            srv.replay([job(10)], [0.0])
        assert e.value.code == 1
        drain_all(srv)
        recs, _ = srv.replay([], [])
        assert recs == []


def test_age_priority_ranks_follow_admission_order():
    """Under VP_SERVE_AGE_PRIORITY a job admitted while others run takes the
    rank below the youngest running job's (0 when the server is idle), capped
    at the lowest of the modelled levels; FCFS reports rank 0."""
    with vp.Server(1 << 30, lanes=8, fake=True) as srv:
        recs, _ = srv.replay([job(5000) for _ in range(3)], [0.0, 0.1, 0.2])
        assert [r[4] for r in recs] == [0, 0, 0]
        srv.set_policy(vp.VP_SERVE_AGE_PRIORITY)
        # eight overlapping 5 ms jobs, then one after everything has finished
        arr = [0.1 * i for i in range(8)] + [40.0]
        recs, _ = srv.replay([job(5000) for _ in arr], arr)
        assert [r[4] for r in recs] == [0, 1, 2, 3, 4, 5, 5, 5, 0]
        srv.submit(job(20000))
        with pytest.raises(vp.VPError):                 # not while a job runs
            srv.set_policy(vp.VP_SERVE_FCFS)
        drain_all(srv)
        srv.set_policy(vp.VP_SERVE_FCFS)
        with pytest.raises(vp.VPError):
            srv.set_policy(2)


def test_replay_invariants_random_traces():
    """Random traces on the fake server (sizes, arrivals, lanes, pool): every
    job is reported once and in trace order; admission is first come, first
    served (admission times never decrease along the trace); a job never
    starts before it was submitted; its run lasts its C microseconds; the
    server never runs more jobs than lanes, nor uses more pool than it has."""
    import random
    unit = per_channel_bytes()
    rng = random.Random(2602)
    for trial in range(6):
        lanes = rng.choice([1, 2, 3, 5])
        pool = (rng.choice([3000, 6000, 20000]) * unit) + (1 << 20)
        n = rng.randint(5, 25)
        sizes = [rng.randint(50, 2500) for _ in range(n)]
        arr, t = [], 0.0
        for _ in range(n):
            t += rng.choice([0.0, 0.05, 0.3, 1.0])
            arr.append(round(t, 3))
        with vp.Server(pool, lanes=lanes, fake=True) as srv:
            recs, sub = srv.replay([job(C) for C in sizes], arr, timeout_s=30.0)
            st = srv.stats()
        assert [r[0] for r in recs] == list(range(recs[0][0], recs[0][0] + n))
        assert all(r[1] == 0 for r in recs)
        admits = [r[2] for r in recs]
        assert all(b >= a - 0.05 for a, b in zip(admits, admits[1:])), (trial, admits)
        for r, s_ms, C in zip(recs, sub, sizes):
            assert r[2] >= s_ms - 1e-3
            assert r[3] - r[2] == pytest.approx(C * 1e-3, abs=0.5)
        assert 1 <= st["max_in_flight"] <= lanes
        assert st["pool_high_water"] <= pool and st["pool_used"] == 0
        # at any instant at most `lanes` jobs ran
        events = sorted([(r[2], 1) for r in recs] + [(r[3], -1) for r in recs], key=lambda e: (e[0], e[1]))
        live = 0
        for _, d in events:
            live += d
            assert live <= lanes
