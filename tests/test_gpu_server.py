"""The job server (vp_server_*): jobs admitted by lane and pool memory while
others run, their kernels overlapping on several streams. Every job's
outputs must be the same in the mix as alone (the plan path on the same
inputs: the same kernels, so equal to the bit), and one job is compared with
the oracle directly.
"""
import numpy as np
import pytest
import torch

import paper_2602_12098_gb300 as vp
from paper_2602_12098_gb300 import workloads as W
from vp_gpu_util import assert_parity, compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vp.load()


SHAPES = [  # K, M, qam, n, lam, demap, frac
    (4, 8, 16, 16, 0.0, 0, 0), (8, 8, 64, 64, 0.0, 0, 0), (16, 16, 256, 256, 0.0, 0, 0),
    (12, 16, 64, 128, 0.0, 0, 0), (8, 4, 4, 32, 0.6, 0, 0), (16, 16, 256, 64, 0.0, 1, 0),
    (8, 8, 64, 64, 0.0, 0, 11), (2, 2, 16, 81, 0.0, 0, 0),
]


class JobData:
    def __init__(self, i, shape, dev):
        K, M, qam, n, lam, demap, frac = shape
        rng = W.rng_for(120, i)
        self.shape = shape
        self.C = int(rng.integers(20, 400))
        self.S = 14
        self.Hn = W.channels(rng, self.C, K, M)
        self.sn = W.symbols(rng, self.C * self.S, K, qam)
        self.H = torch.from_numpy(self.Hn).to(dev)
        self.sym = torch.from_numpy(self.sn).to(dev)
        V = self.C * self.S
        self.x = torch.full((V, M), complex(np.nan, np.nan), dtype=torch.complex64, device=dev)
        self.l = torch.full((V, K, 2), 99, dtype=torch.int8, device=dev)
        self.g = torch.full((V,), np.nan, dtype=torch.float32, device=dev)
        self.st = torch.full((self.C,), 255, dtype=torch.uint8, device=dev)

    def desc(self, ready_event=None):
        K, M, qam, n, lam, demap, frac = self.shape
        return vp.job_desc(K, M, qam, n, self.C, self.S, self.H, self.sym, self.x, self.l, self.g, self.st, lam=lam,
                           demap=demap, frac_bits=frac, ready_event=ready_event)

    def outputs(self):
        return (self.x.cpu().numpy(), self.l.cpu().numpy(), self.g.cpu().numpy(), self.st.cpu().numpy())

    def alone(self):
        K, M, qam, n, lam, demap, frac = self.shape
        V = self.C * self.S
        dev = self.H.device
        x = torch.empty((V, M), dtype=torch.complex64, device=dev)
        l = torch.empty((V, K, 2), dtype=torch.int8, device=dev)
        g = torch.empty((V,), dtype=torch.float32, device=dev)
        st = torch.empty((self.C,), dtype=torch.uint8, device=dev)
        with vp.Plan(K, M, qam, n, lam=lam, demap=demap, frac_bits=frac) as plan:
            vp.vp_factorize(plan.handle, self.H, self.C, None, None, None, st)
            vp.vp_precode(plan.handle, self.sym, self.S, None, V, x, l, g)
            torch.cuda.synchronize()
        return (x.cpu().numpy(), l.cpu().numpy(), g.cpu().numpy(), st.cpu().numpy())


def _state_bytes(C, K, M, n):
    return C * (24 * K * K + 16 * K * M + 20 * n + 5 * K + 300)


def test_jobs_same_alone_and_in_the_mix():
    dev = torch.device("cuda:0")
    jobs = [JobData(i, SHAPES[i % len(SHAPES)], dev) for i in range(40)]
    # a pool that holds only a few of the larger jobs at once: admission waits for memory
    pool = 3 * _state_bytes(400, 16, 16, 256)
    with vp.Server(pool, lanes=4) as srv:
        ids = {}
        reported = {}
        for i, jd in enumerate(jobs):
            ids[srv.submit(jd.desc())] = i
            if i % 3 == 2:                 # some arrive while others run
                for rec in srv.poll():
                    reported[rec[0]] = rec
        srv.drain(120.0)
        for rec in srv.poll():
            reported[rec[0]] = rec
        st = srv.stats()
    assert sorted(reported) == sorted(ids)
    assert st["completed"] == st["submitted"] == len(jobs) and st["queued"] == 0 and st["in_flight"] == 0
    assert 1 < st["max_in_flight"] <= 4
    assert st["pool_high_water"] <= pool and st["pool_used"] == 0
    for k, (jid, status, t0, t1, rank) in reported.items():
        assert status == 0 and 0.0 <= t0 <= t1, reported[k]
    for jd in jobs:
        mix, alone = jd.outputs(), jd.alone()
        for a, b in zip(mix, alone):
            assert np.array_equal(a, b), jd.shape


def test_job_in_the_mix_matches_the_oracle(orc):
    dev = torch.device("cuda:0")
    jobs = [JobData(100 + i, SHAPES[i % 3], dev) for i in range(6)]
    with vp.Server(64 << 20, lanes=3) as srv:
        for jd in jobs:
            srv.submit(jd.desc())
        srv.drain(60.0)
    jd = jobs[1]                                       # 8 x 8, 64-QAM, n = 64
    K, M, qam, n = jd.shape[:4]
    x, l, g, stt = jd.outputs()
    off = W.vec_offsets_uniform(jd.C, jd.S)
    ref = orc.precode_batch(jd.Hn, jd.sn, off, qam, n, nthreads=orc.max_threads())
    gpu = {"x": x, "l": l, "gamma": g.astype(np.float64)}
    assert np.array_equal(stt & 3, ref["status"])
    assert_parity(compare(orc, jd.Hn, jd.sn, off, qam, gpu, ref))


def test_ready_event_orders_the_inputs():
    """A job whose inputs are written on another stream waits for them."""
    dev = torch.device("cuda:0")
    jd = JobData(200, SHAPES[2], dev)
    want = jd.alone()
    side = torch.cuda.Stream(device=dev)
    Hsrc = jd.H.clone()
    jd.H.zero_()
    torch.cuda.synchronize()
    ev = torch.cuda.Event()
    with torch.cuda.stream(side):
        torch.cuda._sleep(2_000_000)               # the copy lands well after the submission
        jd.H.copy_(Hsrc)
        ev.record(side)
    with vp.Server(64 << 20, lanes=2) as srv:
        srv.submit(jd.desc(ready_event=ev))
        srv.drain(60.0)
    for a, b in zip(jd.outputs(), want):
        assert np.array_equal(a, b)


def test_job_larger_than_the_pool_is_refused():
    dev = torch.device("cuda:0")
    jd = JobData(300, SHAPES[2], dev)
    with vp.Server(1 << 20, lanes=1) as srv:
        with pytest.raises(vp.VPError) as e:
            srv.submit(jd.desc())
        assert e.value.code == 6
        assert srv.stats()["submitted"] == 0


def test_drain_deadline_returns_timeout_then_completes():
    """vp_server_drain with a deadline shorter than the work returns
    VP_ERR_TIMEOUT (the jobs keep running); a longer one then completes."""
    dev = torch.device("cuda:0")
    jobs = [JobData(400 + i, SHAPES[2], dev) for i in range(6)]
    side = torch.cuda.Stream(device=dev)
    ev = torch.cuda.Event()
    with torch.cuda.stream(side):
        torch.cuda._sleep(50_000_000)              # holds the first job's inputs for ~25 ms
        ev.record(side)
    with vp.Server(256 << 20, lanes=2) as srv:
        srv.submit(jobs[0].desc(ready_event=ev))
        for jd in jobs[1:]:
            srv.submit(jd.desc())
        with pytest.raises(vp.VPError) as e:
            srv.drain(0.0)
        assert e.value.code == 4
        srv.drain(60.0)
        done = srv.poll()
        assert len(done) == len(jobs) and all(rec[1] == 0 for rec in done)
        st = srv.stats()
        assert st["completed"] == len(jobs) and st["in_flight"] == 0 and st["queued"] == 0
    for jd in jobs[:2]:
        for a, b in zip(jd.outputs(), jd.alone()):
            assert np.array_equal(a, b)


def test_replay_under_age_priority_same_as_alone():
    """A trace replayed under VP_SERVE_AGE_PRIORITY (jobs on streams of
    several priorities, overlapping): every job's outputs equal the plan
    path's, jobs admitted while others run rank below them, and each job is
    submitted no earlier than its arrival time."""
    dev = torch.device("cuda:0")
    jobs = [JobData(500 + i, SHAPES[i % len(SHAPES)], dev) for i in range(16)]
    arrival = [0.05 * i for i in range(len(jobs))]
    with vp.Server(256 << 20, lanes=4) as srv:
        srv.set_policy(vp.VP_SERVE_AGE_PRIORITY)
        recs, sub = srv.replay([jd.desc() for jd in jobs], arrival, timeout_s=120.0)
        st = srv.stats()
    assert st["completed"] == len(jobs) and st["max_in_flight"] > 1
    for r, a, s in zip(recs, arrival, sub):
        assert r[1] == 0 and s >= a and 0.0 <= r[2] <= r[3]
    assert recs[0][4] == 0 and max(r[4] for r in recs) > 0
    for jd in jobs:
        for a, b in zip(jd.outputs(), jd.alone()):
            assert np.array_equal(a, b), jd.shape
