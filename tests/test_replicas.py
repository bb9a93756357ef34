"""Multi-process path of bench.py: one independent problem per rank (replicas).

Run as two gloo ranks on the CPU: the job time must be the slowest rank's and
the work the sum of every rank's particles; ranks get different seeds.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, n = bench.reduce_over_ranks(10.0 + 5.0 * rank, 1000 * (rank + 1))
    w = bench.workload_for(rank, 2048)
    q.put((rank, t, n, float(w.pos[0, 0])))
    dist.destroy_process_group()


def test_replica_aggregation_gloo_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, n, x0 in res:
        assert t == 15.0 and n == 3000
    assert res[0][3] != res[1][3]          # independent problems per rank
