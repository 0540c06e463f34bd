"""The host side of the domain-decomposed hop on CPU processes (gloo): the
time-slab and z x t grid geometry, the neighbours and global boundary signs,
and the face exchange of DistributedExchange with 2 and 4 ranks (along t, and
along z and t on a 2 x 2 grid), whose routing must give every domain the
`to_prev` face of its next domain along each direction and the `to_next` face
of its previous one (with two ranks both are the same peer), and the hooks of
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


def _grid_worker(rank, world, port, L, nz, nt, errq):
    """One rank of a 2 x 2 grid: every face carries its sender, direction and
    kind, and after DistributedComm.exchange each rank must hold its z and t
    neighbours' faces; the leading-bytes form moves only those bytes."""
    import torch.distributed as dist
    try:
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        g = dd.DomainGrid(L, nz, nt, antiperiodic_t=True)
        n = 64

        def tag(r, mu, kind):
            return 1000.0 * r + 10.0 * mu + kind

        faces = []
        for mu in g.dirs:
            faces += [torch.full((n,), tag(rank, mu, 1), dtype=torch.float64),
                      torch.full((n,), tag(rank, mu, 2), dtype=torch.float64),
                      torch.zeros(n, dtype=torch.float64), torch.zeros(n, dtype=torch.float64)]
        comm = dd.DistributedComm(g, rank, tuple(faces))
        comm.exchange()
        for k, mu in enumerate(g.dirs):
            nxt, prv = g.next(rank, mu), g.prev(rank, mu)
            assert bool((faces[4 * k + 2] == tag(nxt, mu, 1)).all()), (rank, mu, faces[4 * k + 2][:2])
            assert bool((faces[4 * k + 3] == tag(prv, mu, 2)).all()), (rank, mu, faces[4 * k + 3][:2])
        for k in range(len(g.dirs)):
            faces[4 * k + 2].fill_(-1.0)
            faces[4 * k + 3].fill_(-1.0)
        comm.exchange(16 * 8, 8 * 8)  # t: 16 words, z: 8 words
        for k, mu in enumerate(g.dirs):
            m = 16 if mu == dd.T_DIR else 8
            assert bool((faces[4 * k + 2][:m] == tag(g.next(rank, mu), mu, 1)).all()), (rank, mu)
            assert bool((faces[4 * k + 2][m:] == -1.0).all()), (rank, mu)
            assert bool((faces[4 * k + 3][:m] == tag(g.prev(rank, mu), mu, 2)).all()), (rank, mu)
        dz, dt = g.coords(rank)
        assert g.negate_to_prev(rank, dd.T_DIR) == (dt == 0) and not g.negate_to_prev(rank, dd.Z_DIR)
        assert g.negate_to_next(rank, dd.T_DIR) == (dt == nt - 1) and not g.negate_to_next(rank, dd.Z_DIR)
        dist.barrier()
        dist.destroy_process_group()
    except Exception as e:  # reported to the parent
        errq.put(f"rank {rank}: {e!r}")


@pytest.mark.parametrize("nz,nt", [(2, 2), (4, 1)])
def test_grid_exchange_routes_z_and_t_faces(nz, nt):
    world = nz * nt
    L = (4, 4, 8, 8)
    ctx = mp.get_context("spawn")
    errq = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_grid_worker, args=(r, world, port, L, nz, nt, errq)) for r in range(world)]
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


def test_domain_grid_geometry():
    """The z x t grid: local extents, every site in exactly one domain, the
    sites of each block having z and t in the domain's ranges and listed in
    the domain's own lexicographic order, the neighbours along z and t."""
    L = (2, 4, 6, 8)
    V = int(np.prod(L))
    idx = np.arange(V)
    x = idx % L[0]
    y = (idx // L[0]) % L[1]
    z = (idx // (L[0] * L[1])) % L[2]
    t = idx // (L[0] * L[1] * L[2])
    for nz, nt in ((1, 1), (3, 1), (1, 4), (3, 2), (3, 4)):
        g = dd.DomainGrid(L, nz, nt, antiperiodic_t=True)
        assert g.local_L == (2, 4, 6 // nz, 8 // nt) and g.ndomains == nz * nt
        seen = np.zeros(V, dtype=int)
        for d in range(g.ndomains):
            b = idx[g.block(d)]
            seen[b] += 1
            dz, dt = g.coords(d)
            assert np.all(z[b] // g.lz == dz) and np.all(t[b] // g.lt == dt)
            # local lexicographic order: x fastest, then y, local z, local t
            loc = x[b] + L[0] * (y[b] + L[1] * ((z[b] - dz * g.lz) + g.lz * (t[b] - dt * g.lt)))
            assert np.array_equal(loc, np.arange(g.local_volume))
            assert g.next(g.prev(d, dd.Z_DIR), dd.Z_DIR) == d and g.next(g.prev(d, dd.T_DIR), dd.T_DIR) == d
            assert g.coords(g.next(d, dd.Z_DIR)) == ((dz + 1) % nz, dt)
            assert g.coords(g.next(d, dd.T_DIR)) == (dz, (dt + 1) % nt)
        assert np.all(seen == 1)
        assert g.dirs == ((dd.T_DIR, dd.Z_DIR) if nz > 1 else (dd.T_DIR,))
    for bad in ((4, 1), (6, 1), (1, 3)):  # 6/4 not integral; Lz/6 = 1; Lt/3 not integral
        with pytest.raises(ValueError):
            dd.DomainGrid(L, *bad)
