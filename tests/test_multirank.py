"""N > 1 host logic of bench.py on CPU (gloo, world size 2): replicas only.

Each rank runs its own population (distinct instance ids, same seed, so
independent Philox streams) and the job's time is the slowest rank's while
the work is summed over ranks.  No GPU is used: the aggregation runs over
gloo on CPU tensors, the same code path bench.py takes over NCCL.
"""
from __future__ import annotations

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, work = bench.aggregate(dist, ms=10.0 + 5.0 * rank, work=1000.0 * (rank + 1), device="cpu")
    wl = bench.rank_workload(rank, 1 << 21)
    out[rank] = (ms, work, wl["instance_id"], wl["seed"], wl["R0"])
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_time_sum_work_distinct_instances():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][:2] == (15.0, 3000.0) and res[1][:2] == (15.0, 3000.0)
    assert {res[0][2], res[1][2]} == {0, 1}
    assert res[0][3] == res[1][3] and res[0][4] == res[1][4] == 1 << 21


def test_single_process_aggregate_is_identity():
    import bench
    assert bench.aggregate(None, 3.5, 7.0, "cpu") == (3.5, 7.0)
