"""The host side of the domain-decomposed hop on CPU processes (gloo): the
time-slab geometry, the neighbours and global boundary signs, and the face
exchange of DistributedExchange with 2 and 4 ranks, whose routing must give
every domain the `to_prev` face of its next domain and the `to_next` face of
its previous one (with two ranks both are the same peer), and the hooks of
the domain-decomposed solver (DistributedComm: the same exchange, of the
whole buffers or of their leading bytes, and the sum of host values over the
ranks).  The GPU kernels of the hop and the solver
are checked against the oracle in tests/test_gpu_dd.py."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_1209_5942_gb300 import dd


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, L, errq):
    import torch.distributed as dist
    try:
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        slabs = dd.TimeSlabs(L, world, antiperiodic_t=True)
        n = 96
        # faces tagged with the sender and the face kind
        to_prev = torch.full((n,), 100.0 * rank + 1.0, dtype=torch.float64)
        to_next = torch.full((n,), 100.0 * rank + 2.0, dtype=torch.float64)
        to_prev[::7] = -rank  # some structure inside the buffer
        from_next = torch.zeros(n, dtype=torch.float64)
        from_prev = torch.zeros(n, dtype=torch.float64)
        for _ in range(3):  # repeated exchanges stay matched
            dd.DistributedExchange().exchange(slabs, rank, to_prev, to_next, from_next, from_prev)
        nxt, prv = (rank + 1) % world, (rank - 1) % world
        exp_next = torch.full((n,), 100.0 * nxt + 1.0, dtype=torch.float64)
        exp_next[::7] = -nxt
        exp_prev = torch.full((n,), 100.0 * prv + 2.0, dtype=torch.float64)
        assert torch.equal(from_next, exp_next), (rank, from_next[:3])
        assert torch.equal(from_prev, exp_prev), (rank, from_prev[:3])
        # the solver's hooks: the same routing, and sums over the ranks
        comm = dd.DistributedComm(slabs, rank, (to_prev, to_next, from_next, from_prev))
        from_next.zero_()
        from_prev.zero_()
        comm.exchange()
        assert torch.equal(from_next, exp_next) and torch.equal(from_prev, exp_prev), rank
        # a face of a lower format: only the leading bytes move, the rest of
        # the receive buffers is left as it was
        from_next.fill_(-7.0)
        from_prev.fill_(-7.0)
        comm.exchange(40 * 8)
        assert torch.equal(from_next[:40], exp_next[:40]) and torch.equal(from_prev[:40], exp_prev[:40]), rank
        assert bool((from_next[40:] == -7.0).all()) and bool((from_prev[40:] == -7.0).all()), rank
        sums = comm.allreduce([float(rank + 1), 0.5, -2.0 * rank])
        assert sums == [world * (world + 1) / 2, 0.5 * world, -float(world * (world - 1))], (rank, sums)
        assert slabs.next(rank) == nxt and slabs.prev(rank) == prv
        assert slabs.negate_to_prev(rank) == (rank == 0)
        assert slabs.negate_to_next(rank) == (rank == world - 1)
        dist.barrier()
        dist.destroy_process_group()
    except Exception as e:  # reported to the parent
        errq.put(f"rank {rank}: {e!r}")


@pytest.mark.parametrize("world", [2, 4])
def test_face_exchange_routes_faces_to_the_neighbours(world):
    L = (4, 4, 4, 16)
    ctx = mp.get_context("spawn")
    errq = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, L, errq)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
    errs = []
    while not errq.empty():
        errs.append(errq.get())
    assert not alive, "a rank did not finish"
    assert not errs, errs
    assert all(p.exitcode == 0 for p in procs)


def test_time_slab_geometry():
    """Local extents, the contiguous lexicographic blocks, and the sites of
    each block having t in the domain's range (t is the slowest index)."""
    L = (4, 2, 6, 12)
    for nt in (1, 2, 3, 6):
        s = dd.TimeSlabs(L, nt, antiperiodic_t=False)
        assert s.local_L == (4, 2, 6, 12 // nt)
        V = int(np.prod(L))
        idx = np.arange(V)
        t = idx // (L[0] * L[1] * L[2])
        for d in range(nt):
            b = idx[s.block(d)]
            assert np.all(t[b] // s.lt == d)
            assert len(b) == s.local_volume
        assert not s.negate_to_prev(0) and not s.negate_to_next(nt - 1)
    for bad in (5, 4, 12 * 2):  # 12/5 not integral; 12/4 = 3 odd; 12/24 < 2
        with pytest.raises(ValueError):
            dd.TimeSlabs(L, bad)


def test_single_domain_exchange_is_a_local_copy():
    s = dd.TimeSlabs((4, 4, 4, 4), 1)
    a, b = torch.arange(8.0), torch.arange(8.0) + 10
    c, e = torch.zeros(8), torch.zeros(8)
    dd.DistributedExchange().exchange(s, 0, a, b, c, e)
    assert torch.equal(c, a) and torch.equal(e, b)
