"""Domain decomposition of the half hop along t: the host side -- geometry,
neighbours, the global boundary sign and the face exchange -- around the
library's ``lqcd_dd_pack`` / ``lqcd_dd_dslash`` (include/lqcd.h).

The paper names a multi-GPU Dslash as its outlook (Sec. 6).  A lattice of
extent Lt is split into nt domains of Lt/nt consecutive t slices.  With the
lexicographic site order t is the slowest coordinate, so a domain's links and
spinors are one contiguous block of the global arrays, and each domain is an
ordinary field of the library on its local geometry.  One half hop is

    pack the two faces of every domain  ->  exchange  ->  the domain hops,

where a face holds the spin-projected half spinors (6 complex per boundary
site of one parity) that a neighbour's boundary t hops need.  The exchange
moves, for every domain d, its ``to_prev`` face to domain d-1 (which uses it
as ``from_next``) and its ``to_next`` face to domain d+1 (``from_prev``).
``LocalExchange`` does this inside one process (all domains on one device,
device copies); ``DistributedExchange`` with one domain per rank of a
``torch.distributed`` group (NCCL for CUDA tensors, gloo for CPU tensors).
The domain-decomposed FP64 CG (``lqcd_dd_cg_solve``) runs every half hop of
its operator this way; its norms are summed over the domains held by the
call and then over processes.  ``cg_solve_local_domains`` holds all domains in
one call (the library moves the faces itself); ``cg_solve_distributed``
holds one domain per rank and gives the library hooks that move the faces
with ``DistributedExchange`` and sum the norms with ``all_reduce``.
Nothing here does arithmetic of the method: every step of the hop and of
the solver runs in the library's kernels.
"""
from __future__ import annotations

import torch

from . import lqcd


class TimeSlabs:
    """nt domains of the lattice L = (Lx, Ly, Lz, Lt), split along t."""

    def __init__(self, L, nt: int, antiperiodic_t: bool = True):
        L = tuple(int(v) for v in L)
        if nt < 1 or L[3] % nt:
            raise ValueError(f"Lt = {L[3]} is not a multiple of nt = {nt}")
        lt = L[3] // nt
        if lt % 2 or lt < 2:
            raise ValueError(f"local extent Lt/nt = {lt} must be even and >= 2 (parities must agree)")
        self.L, self.nt, self.lt = L, nt, lt
        self.antiperiodic_t = bool(antiperiodic_t)

    @property
    def local_L(self):
        return (self.L[0], self.L[1], self.L[2], self.lt)

    @property
    def local_volume(self) -> int:
        return self.L[0] * self.L[1] * self.L[2] * self.lt

    def prev(self, d: int) -> int:
        return (d - 1) % self.nt

    def next(self, d: int) -> int:
        return (d + 1) % self.nt

    def negate_to_prev(self, d: int) -> bool:
        """The first domain's t = 0 slice is the +t neighbour of the last
        domain's t = Lt/nt - 1 slice across the global boundary."""
        return self.antiperiodic_t and d == 0

    def negate_to_next(self, d: int) -> bool:
        return self.antiperiodic_t and d == self.nt - 1

    def block(self, d: int) -> slice:
        """Lexicographic sites of domain d in the global arrays."""
        n = self.local_volume
        return slice(d * n, (d + 1) * n)

    def split(self, a):
        """A global site-major array ([V, ...] or [nrhs, V, ...] with axis=0
        the sites) -> the nt local blocks (views)."""
        return [a[self.block(d)] for d in range(self.nt)]


class LocalExchange:
    """All domains in one process: from_next[d] <- to_prev[d+1] and
    from_prev[d] <- to_next[d-1] by device-to-device copies."""

    def exchange(self, slabs: TimeSlabs, to_prev, to_next, from_next, from_prev):
        for d in range(slabs.nt):
            from_next[d].copy_(to_prev[slabs.next(d)])
            from_prev[d].copy_(to_next[slabs.prev(d)])


class DistributedExchange:
    """One domain per rank (rank = domain index) of a torch.distributed group.
    Each rank sends to_prev to rank d-1 and to_next to rank d+1 and receives
    from_next from d+1 and from_prev from d-1; with two ranks both neighbours
    are the same peer, and the messages are told apart by their order (NCCL)
    and their tags (gloo).  nt = 1 reduces to a local copy."""

    TAG_TO_PREV, TAG_TO_NEXT = 17, 18

    def __init__(self, group=None):
        self.group = group

    def exchange(self, slabs: TimeSlabs, rank: int, to_prev, to_next, from_next, from_prev):
        import torch.distributed as dist
        if slabs.nt == 1:
            from_next.copy_(to_prev)
            from_prev.copy_(to_next)
            return
        p, n = slabs.prev(rank), slabs.next(rank)
        ops = [dist.P2POp(dist.isend, to_prev, p, self.group, self.TAG_TO_PREV),
               dist.P2POp(dist.isend, to_next, n, self.group, self.TAG_TO_NEXT),
               dist.P2POp(dist.irecv, from_next, n, self.group, self.TAG_TO_PREV),
               dist.P2POp(dist.irecv, from_prev, p, self.group, self.TAG_TO_NEXT)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()


def face_buffers(slabs: TimeSlabs, prec: int, device="cuda"):
    """(to_prev, to_next, from_next, from_prev) face buffers of one domain."""
    nb = lqcd.lqcd_dd_face_bytes(slabs.local_L, prec)
    if nb == 0:
        raise ValueError("no face size for this geometry / precision")
    return tuple(torch.empty(nb // 8, dtype=torch.float64, device=device) for _ in range(4))


def dslash_local_domains(ctx, slabs: TimeSlabs, gauges, ins, outs, out_parity, dagger=0, bufs=None):
    """One half hop over all domains of `slabs` held in this process (one
    device): gauges[d] (library fields on the local geometry), ins[d] / outs[d]
    (lqcd_field half fields of domain d).  bufs: per-domain face buffers
    (allocated if None); returns them for reuse."""
    if bufs is None:
        bufs = [face_buffers(slabs, ins[0].prec) for _ in range(slabs.nt)]
    for d in range(slabs.nt):
        lqcd.lqcd_dd_pack(ctx, gauges[d], ins[d], bufs[d][0], bufs[d][1], out_parity, dagger,
                          slabs.negate_to_prev(d), slabs.negate_to_next(d))
    LocalExchange().exchange(slabs, [b[0] for b in bufs], [b[1] for b in bufs], [b[2] for b in bufs],
                             [b[3] for b in bufs])
    for d in range(slabs.nt):
        lqcd.lqcd_dd_dslash(ctx, gauges[d], ins[d], outs[d], bufs[d][2], bufs[d][3], out_parity, dagger)
    return bufs


def dslash_distributed(ctx, slabs: TimeSlabs, rank: int, gauge, inp, out, out_parity, dagger=0, bufs=None,
                       exchange: DistributedExchange | None = None):
    """One half hop of this rank's domain in a torch.distributed job (one
    domain per rank; NCCL moves the CUDA face buffers)."""
    if bufs is None:
        bufs = face_buffers(slabs, inp.prec)
    to_prev, to_next, from_next, from_prev = bufs
    lqcd.lqcd_dd_pack(ctx, gauge, inp, to_prev, to_next, out_parity, dagger, slabs.negate_to_prev(rank),
                      slabs.negate_to_next(rank))
    torch.cuda.current_stream().synchronize()
    (exchange or DistributedExchange()).exchange(slabs, rank, to_prev, to_next, from_next, from_prev)
    lqcd.lqcd_dd_dslash(ctx, gauge, inp, out, from_next, from_prev, out_parity, dagger)
    return bufs


def cg_solve_local_domains(ctx, slabs: TimeSlabs, gauges, bs, xs, kappa, mu, params, faces=None,
                           allow_noconv=False):
    """Domain-decomposed CG (FP64, or mixed with an F32 / float-float inner
    format as params say) with every domain of `slabs` held in this process
    (one device): gauges[d], bs[d], xs[d] (EO full fields of domain d
    on the local geometry).  Returns the solve's stats."""
    if faces is None:
        faces = [face_buffers(slabs, lqcd.LQCD_F64) for _ in range(slabs.nt)]
    return lqcd.lqcd_dd_cg_solve(ctx, gauges, bs, xs, faces, 0, slabs.nt, kappa, mu, params,
                                 antiperiodic_t=slabs.antiperiodic_t, allow_noconv=allow_noconv)


class DistributedComm:
    """The communication hooks of a domain-decomposed solve with one domain
    per rank of a torch.distributed group: exchange(nbytes) moves the leading
    nbytes of this rank's faces (all of them if None; DistributedExchange,
    device faces through host copies for gloo),
    allreduce(values) sums host floats over the group (on the CPU for gloo,
    on the device for NCCL)."""

    def __init__(self, slabs: TimeSlabs, rank: int, faces, group=None):
        self.slabs, self.rank, self.faces, self.group = slabs, rank, faces, group
        self._ex = DistributedExchange(group)

    def exchange(self, nbytes=None):
        import torch.distributed as dist
        faces = self.faces
        if nbytes is not None:  # the face of a lower format fills the buffers' leading bytes
            faces = [f.view(torch.uint8)[:nbytes] for f in faces]
        if faces[0].is_cuda and dist.get_backend(self.group) == "gloo":
            # gloo moves host memory: stage the device faces through the host
            host = [f.cpu() for f in faces]
            self._ex.exchange(self.slabs, self.rank, *host)
            faces[2].copy_(host[2])
            faces[3].copy_(host[3])
        else:
            self._ex.exchange(self.slabs, self.rank, *faces)
        if faces[0].is_cuda:
            torch.cuda.current_stream().synchronize()

    def allreduce(self, values):
        import torch.distributed as dist
        cpu = dist.get_backend(self.group) == "gloo"
        t = torch.tensor(list(values), dtype=torch.float64, device="cpu" if cpu else self.faces[0].device)
        dist.all_reduce(t, group=self.group)
        return t.tolist()


def cg_solve_distributed(ctx, slabs: TimeSlabs, rank: int, gauge, b, x, kappa, mu, params, group=None,
                         faces=None, allow_noconv=False):
    """Domain-decomposed CG (FP64 or mixed, as params say) with this rank's
    domain (rank = domain index) in a torch.distributed job; NCCL moves the
    CUDA face buffers."""
    if faces is None:
        faces = face_buffers(slabs, lqcd.LQCD_F64)
    comm = DistributedComm(slabs, rank, faces, group)
    return lqcd.lqcd_dd_cg_solve(ctx, [gauge], [b], [x], [faces], rank, slabs.nt, kappa, mu, params,
                                 antiperiodic_t=slabs.antiperiodic_t, exchange=comm.exchange,
                                 allreduce=comm.allreduce, allow_noconv=allow_noconv)
