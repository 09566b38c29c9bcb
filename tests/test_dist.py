"""Multi-process host logic of bench.py on CPU (gloo, world size 2): each
rank solves its own seeded replica, and the whole-job figures are the max
over ranks of the time and the sum over ranks of the work.  No GPU."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    seed = bench.replica_seed(r)
    u0 = W.initial_condition(W.config(bench.WORKLOAD, seed=seed))
    t_local = 1.0 + rank          # rank 1 is the slowest
    work_local = 100.0 * (rank + 1)
    t, w = bench.aggregate(t_local, work_local, dist, "cpu")
    out[rank] = (t, w, float(u0[0, 0]), seed)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_aggregate_max_time_and_summed_work():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        ps = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in ps:
            p.start()
        for p in ps:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.0           # max over ranks
    assert res[0][1] == res[1][1] == 300.0         # sum over ranks
    assert res[0][3] != res[1][3]                  # distinct replicas
    assert res[0][2] != res[1][2]


def test_single_process_aggregate_is_identity():
    import bench
    assert bench.aggregate(1.5, 7.0) == (1.5, 7.0)
