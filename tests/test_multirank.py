"""Multi-rank path of bench.py on the CPU (gloo, world size 2): every rank runs
its own replica (the single case does not shard; replicas only), the timed
region is the maximum over ranks, and the value counts all ranks' cells."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t = bench.reduce_times(0.5 + rank, dist)
    v = bench.whole_job_value(1000, 10, world, t)
    out[rank] = (t, v)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_reduce_max_time_and_sum_cells():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (1.5, 2 * 1000 * 10 / 1.5)
