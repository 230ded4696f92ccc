"""Host-side logic of the multi-GPU benchmark (replicas, weak scaling) on CPU gloo ranks:
the job time is the maximum over ranks and every rank sees the same value."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t = bench.job_time(1.0 + 0.5 * rank, world)
    out[rank] = t
    dist.barrier()
    dist.destroy_process_group()


def test_job_time_is_max_over_ranks():
    import torch.multiprocessing as mp

    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1] == 1.5


def test_single_rank_job_time():
    import bench

    assert bench.job_time(2.5, 1) == 2.5
