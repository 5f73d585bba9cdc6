"""Multi-GPU runs are independent replicas: the host logic of bench.py's
N > 1 path (per-rank inputs, slowest-rank time, whole-job rate) on two gloo
ranks on the CPU."""
import os
import socket
import sys

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    from paper_2602_12098_gb300 import workloads as W
    b = bench.replica_batch(W.SMALL_4x4, rank)
    local_s = 1.0 + 0.5 * rank                          # rank 1 is the slow one
    slowest = bench.max_over_ranks(local_s, dist)
    rate = bench.whole_job_rate(ws, b.sym.shape[0], 10, slowest)
    q.put((rank, float(np.abs(b.H).sum()), b.sym.shape[0], slowest, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, h0, v0, s0, rate0), (r1, h1, v1, s1, rate1) = res
    assert h0 != h1                                      # each rank draws its own slot
    assert v0 == v1 == 64                                # same work per rank (weak scaling)
    assert s0 == s1 == 1.5                               # both report the slowest rank
    assert rate0 == rate1 == 2 * 64 * 10 / 1.5


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.0, None) == 2.0
    assert bench.whole_job_rate(1, 100, 5, 2.0) == 250.0
