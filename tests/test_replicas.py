"""Replica aggregation of bench.py across ranks (world size 2, gloo on CPU).

With N GPUs the benchmark runs N independent replicas: each rank reports its
own work and time, the job's value is the sum of the work over the max of the
times.  This checks that host logic without a GPU."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    units, secs = bench.aggregate(1000.0 * (rank + 1), 0.5 + rank, 2)
    out.put((rank, units, secs))
    bench.barrier(2)
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get() for _ in range(2))
    for rank, units, secs in got:
        assert units == 3000.0 and secs == 1.5
