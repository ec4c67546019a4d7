"""The multi-GPU path is replicas only (each rank advances its own seeded
instance; the scheme's work does not shard across ranks here): the one
collective is the max over ranks of the timed seconds.  These tests run that
host-side logic with the gloo backend on CPU, world size 2."""

import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env() == (ws, rank, rank)
        slowest = bench.max_over_ranks(1.0 + rank, device="cpu")
        dist.barrier()
        u = bench.workload(rank)
        out.put((rank, slowest, float(np.abs(u).sum())))
    finally:
        dist.destroy_process_group()


def test_two_replicas_agree_on_the_slowest_time_and_differ_in_data():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(ws))
    assert [r[1] for r in res] == [2.0, 2.0]          # both ranks see the slowest rank
    assert res[0][2] != res[1][2]                    # each rank its own seeded instance


def test_job_value_is_weak_scaling():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_value(1, 1000, 2.0) == 500.0
    assert bench.job_value(4, 1000, 2.0) == 2000.0   # 4 replicas, same time: 4x the units
    assert bench.max_over_ranks(3.5) == 3.5          # no process group: the rank's own time
