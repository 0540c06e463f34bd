"""The N > 1 path of bench.py (independent replicas, one process per GPU) on the
CPU: two gloo ranks reduce their timings and counted bytes the way the GPU run
does (max of the times, sum of the bytes), and the rank environment is read
from the launcher's variables."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world)})
    import bench
    r, lr, w = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        t, b = bench.reduce_over_ranks(dist, 1.0 + rank, 10.0 * (rank + 1), "cpu")
        out[rank] = (r, lr, w, t, b)
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_gpu_run():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        r, lr, w, t, b = out[rank]
        assert (r, lr, w) == (rank, rank, world)
        assert t == 2.0          # the slowest replica sets the time
        assert b == 30.0         # work of all replicas


def test_single_process_needs_no_collective():
    import bench
    assert bench.reduce_over_ranks(None, 1.5, 7.0, "cpu") == (1.5, 7.0)
