"""Domain decomposition of the half hop along t, and along z as well: the host
side -- geometry, neighbours, the global boundary sign and the face exchange
-- around the library's ``lqcd_dd_pack_dir`` / ``lqcd_dd_dslash_zt``
(include/lqcd.h).

The paper names a multi-GPU Dslash as its outlook (Sec. 6).  A lattice is
split into a grid of nz x nt domains, domain d = dz + nz dt holding
Lz/nz consecutive z slices and Lt/nt consecutive t slices; each domain is an
ordinary field of the library on its local geometry (Lx, Ly, Lz/nz, Lt/nt).
With nz = 1 (``TimeSlabs``) t is the slowest lexicographic coordinate, so a
domain's links and spinors are one contiguous block of the global arrays;
with nz > 1 a domain gathers Lt/nt blocks of Lz/nz slices.  One half hop is

    pack the faces of every domain  ->  exchange  ->  the domain hops,

where a face holds the spin-projected half spinors (6 complex per boundary
site of one parity) that a neighbour's boundary hops along t (or z) need.
The exchange moves, for every domain and each split direction, its
``to_prev`` face to the previous domain along that direction (which uses it
as ``from_next``) and its ``to_next`` face to the next one (``from_prev``).
``LocalExchange`` does this inside one process (all domains on one device,
device copies); ``DistributedExchange`` with one domain per rank of a
``torch.distributed`` group (NCCL for CUDA tensors, gloo for CPU tensors).
The domain-decomposed CG (``lqcd_dd_cg_solve``) runs every half hop of its
operator this way; its norms are summed over the domains held by the call
and then over processes.  ``cg_solve_local_domains`` holds all domains in one
call (the library moves the faces itself); ``cg_solve_distributed`` holds one
domain per rank and gives the library hooks that move the faces with
``DistributedExchange`` and sum the norms with ``all_reduce``.  Nothing here
does arithmetic of the method: every step of the hop and of the solver runs
in the library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lqcd

T_DIR, Z_DIR = 3, 2  # the split directions (the library's mu)


class DomainGrid:
    """nz x nt domains of the lattice L = (Lx, Ly, Lz, Lt), split along z and
    t; domain d = dz + nz dt."""

    def __init__(self, L, nz: int, nt: int, antiperiodic_t: bool = True):
        L = tuple(int(v) for v in L)
        for name, n, ext in (("z", nz, L[2]), ("t", nt, L[3])):
            if n < 1 or ext % n:
                raise ValueError(f"L{name} = {ext} is not a multiple of n{name} = {n}")
            loc = ext // n
            if n > 1 and (loc % 2 or loc < 2):
                raise ValueError(f"local extent L{name}/n{name} = {loc} must be even and >= 2 "
                                 "(parities must agree)")
        self.L, self.nz, self.nt = L, nz, nt
        self.lz, self.lt = L[2] // nz, L[3] // nt
        self.antiperiodic_t = bool(antiperiodic_t)

    @property
    def ndomains(self) -> int:
        return self.nz * self.nt

    @property
    def local_L(self):
        return (self.L[0], self.L[1], self.lz, self.lt)

    @property
    def local_volume(self) -> int:
        return self.L[0] * self.L[1] * self.lz * self.lt

    @property
    def dirs(self):
        """The split directions whose faces a half hop exchanges (t first)."""
        return (T_DIR, Z_DIR) if self.nz > 1 else (T_DIR,)

    def coords(self, d: int):
        return d % self.nz, d // self.nz

    def neighbour(self, d: int, mu: int, step: int) -> int:
        dz, dt = self.coords(d)
        if mu == T_DIR:
            dt = (dt + step) % self.nt
        else:
            dz = (dz + step) % self.nz
        return dz + self.nz * dt

    def prev(self, d: int, mu: int = T_DIR) -> int:
        return self.neighbour(d, mu, -1)

    def next(self, d: int, mu: int = T_DIR) -> int:
        return self.neighbour(d, mu, +1)

    def negate_to_prev(self, d: int, mu: int = T_DIR) -> bool:
        """The first t domain's t = 0 slice is the +t neighbour of the last
        one's t = Lt/nt - 1 slice across the global boundary (z is periodic)."""
        return mu == T_DIR and self.antiperiodic_t and self.coords(d)[1] == 0

    def negate_to_next(self, d: int, mu: int = T_DIR) -> bool:
        return mu == T_DIR and self.antiperiodic_t and self.coords(d)[1] == self.nt - 1

    def block(self, d: int):
        """Lexicographic sites of domain d in the global arrays, in the
        domain's own lexicographic order (a slice when nz = 1)."""
        dz, dt = self.coords(d)
        if self.nz == 1:
            n = self.local_volume
            return slice(dt * n, (dt + 1) * n)
        idx = np.arange(int(np.prod(self.L))).reshape(self.L[3], self.L[2], self.L[1] * self.L[0])
        return idx[dt * self.lt:(dt + 1) * self.lt, dz * self.lz:(dz + 1) * self.lz].reshape(-1)

    def split(self, a):
        """A global site-major array ([V, ...]) -> the local blocks (views
        when nz = 1, copies otherwise)."""
        return [a[self.block(d)] for d in range(self.ndomains)]


class TimeSlabs(DomainGrid):
    """nt domains of the lattice L = (Lx, Ly, Lz, Lt), split along t only."""

    def __init__(self, L, nt: int, antiperiodic_t: bool = True):
        super().__init__(L, 1, nt, antiperiodic_t)


class LocalExchange:
    """All domains in one process: along mu, from_next[d] <- to_prev[next(d)]
    and from_prev[d] <- to_next[prev(d)] by device-to-device copies."""

    def exchange(self, slabs: DomainGrid, to_prev, to_next, from_next, from_prev, mu: int = T_DIR):
        for d in range(slabs.ndomains):
            from_next[d].copy_(to_prev[slabs.next(d, mu)])
            from_prev[d].copy_(to_next[slabs.prev(d, mu)])


class DistributedExchange:
    """One domain per rank (rank = domain index) of a torch.distributed group.
    Along mu each rank sends to_prev to the previous domain and to_next to
    the next and receives from_next from the next and from_prev from the
    previous; with two domains along mu both neighbours are the same peer,
    and the messages are told apart by their order (NCCL) and their tags
    (gloo).  One domain along mu reduces to a local copy."""

    TAGS = {T_DIR: (17, 18), Z_DIR: (19, 20)}

    def __init__(self, group=None):
        self.group = group

    def exchange(self, slabs: DomainGrid, rank: int, to_prev, to_next, from_next, from_prev, mu: int = T_DIR):
        import torch.distributed as dist
        p, n = slabs.prev(rank, mu), slabs.next(rank, mu)
        if p == rank:  # one domain along mu
            from_next.copy_(to_prev)
            from_prev.copy_(to_next)
            return
        tag_prev, tag_next = self.TAGS[mu]
        ops = [dist.P2POp(dist.isend, to_prev, p, self.group, tag_prev),
               dist.P2POp(dist.isend, to_next, n, self.group, tag_next),
               dist.P2POp(dist.irecv, from_next, n, self.group, tag_prev),
               dist.P2POp(dist.irecv, from_prev, p, self.group, tag_next)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()


def face_buffers(slabs: DomainGrid, prec: int, device="cuda", mu: int = T_DIR):
    """(to_prev, to_next, from_next, from_prev) face buffers of one domain
    along mu."""
    nb = lqcd.lqcd_dd_face_bytes_dir(slabs.local_L, mu, prec)
    if nb == 0:
        raise ValueError("no face size for this geometry / precision")
    return tuple(torch.empty(nb // 8, dtype=torch.float64, device=device) for _ in range(4))


def domain_faces(slabs: DomainGrid, prec: int, device="cuda"):
    """All face buffers of one domain: the four along t, then (nz > 1) the
    four along z -- the order lqcd_dd_cg_solve takes them in."""
    return tuple(f for mu in slabs.dirs for f in face_buffers(slabs, prec, device, mu))


def dslash_local_domains(ctx, slabs: DomainGrid, gauges, ins, outs, out_parity, dagger=0, bufs=None):
    """One half hop over all domains of `slabs` held in this process (one
    device): gauges[d] (library fields on the local geometry), ins[d] / outs[d]
    (lqcd_field half fields of domain d).  bufs: per-domain face buffers
    (``domain_faces``; allocated if None); returns them for reuse."""
    if bufs is None:
        bufs = [domain_faces(slabs, ins[0].prec) for _ in range(slabs.ndomains)]
    for d in range(slabs.ndomains):
        for k, mu in enumerate(slabs.dirs):
            lqcd.lqcd_dd_pack_dir(ctx, gauges[d], ins[d], mu, bufs[d][4 * k], bufs[d][4 * k + 1], out_parity,
                                  dagger, slabs.negate_to_prev(d, mu), slabs.negate_to_next(d, mu))
    for k, mu in enumerate(slabs.dirs):
        LocalExchange().exchange(slabs, *[[b[4 * k + i] for b in bufs] for i in range(4)], mu=mu)
    for d in range(slabs.ndomains):
        z = bufs[d][6:8] if slabs.nz > 1 else (None, None)
        lqcd.lqcd_dd_dslash_zt(ctx, gauges[d], ins[d], outs[d], bufs[d][2], bufs[d][3], z[0], z[1], out_parity,
                               dagger)
    return bufs


def dslash_distributed(ctx, slabs: DomainGrid, rank: int, gauge, inp, out, out_parity, dagger=0, bufs=None,
                       exchange: DistributedExchange | None = None):
    """One half hop of this rank's domain in a torch.distributed job (one
    domain per rank; NCCL moves the CUDA face buffers)."""
    if bufs is None:
        bufs = domain_faces(slabs, inp.prec)
    for k, mu in enumerate(slabs.dirs):
        lqcd.lqcd_dd_pack_dir(ctx, gauge, inp, mu, bufs[4 * k], bufs[4 * k + 1], out_parity, dagger,
                              slabs.negate_to_prev(rank, mu), slabs.negate_to_next(rank, mu))
    torch.cuda.current_stream().synchronize()
    for k, mu in enumerate(slabs.dirs):
        (exchange or DistributedExchange()).exchange(slabs, rank, *bufs[4 * k:4 * k + 4], mu=mu)
    z = bufs[6:8] if slabs.nz > 1 else (None, None)
    lqcd.lqcd_dd_dslash_zt(ctx, gauge, inp, out, bufs[2], bufs[3], z[0], z[1], out_parity, dagger)
    return bufs


def cg_solve_local_domains(ctx, slabs: DomainGrid, gauges, bs, xs, kappa, mu, params, faces=None,
                           allow_noconv=False):
    """Domain-decomposed CG (FP64, or mixed with an F32 / float-float inner
    format as params say) with every domain of `slabs` held in this process
    (one device): gauges[d], bs[d], xs[d] (EO full fields of domain d on the
    local geometry).  Returns the solve's stats."""
    if faces is None:
        faces = [domain_faces(slabs, lqcd.LQCD_F64) for _ in range(slabs.ndomains)]
    return lqcd.lqcd_dd_cg_solve(ctx, gauges, bs, xs, faces, 0, slabs.nt, kappa, mu, params,
                                 antiperiodic_t=slabs.antiperiodic_t, allow_noconv=allow_noconv, nz=slabs.nz)


class DistributedComm:
    """The communication hooks of a domain-decomposed solve with one domain
    per rank of a torch.distributed group: exchange(t_bytes, z_bytes) moves
    the leading bytes of this rank's t faces and z faces (all of them if
    None; DistributedExchange, device faces through host copies for gloo),
    allreduce(values) sums host floats over the group (on the CPU for gloo,
    on the device for NCCL)."""

    def __init__(self, slabs: DomainGrid, rank: int, faces, group=None):
        self.slabs, self.rank, self.faces, self.group = slabs, rank, faces, group
        self._ex = DistributedExchange(group)

    def exchange(self, t_bytes=None, z_bytes=None):
        import torch.distributed as dist
        for k, mu in enumerate(self.slabs.dirs):
            faces = self.faces[4 * k:4 * k + 4]
            nbytes = t_bytes if mu == T_DIR else z_bytes
            if nbytes is not None:  # the face of a lower format fills the buffers' leading bytes
                faces = [f.view(torch.uint8)[:nbytes] for f in faces]
            if faces[0].is_cuda and dist.get_backend(self.group) == "gloo":
                # gloo moves host memory: stage the device faces through the host
                host = [f.cpu() for f in faces]
                self._ex.exchange(self.slabs, self.rank, *host, mu=mu)
                faces[2].copy_(host[2])
                faces[3].copy_(host[3])
            else:
                self._ex.exchange(self.slabs, self.rank, *faces, mu=mu)
        if self.faces[0].is_cuda:
            torch.cuda.current_stream().synchronize()

    def allreduce(self, values):
        import torch.distributed as dist
        cpu = dist.get_backend(self.group) == "gloo"
        t = torch.tensor(list(values), dtype=torch.float64, device="cpu" if cpu else self.faces[0].device)
        dist.all_reduce(t, group=self.group)
        return t.tolist()


def cg_solve_distributed(ctx, slabs: DomainGrid, rank: int, gauge, b, x, kappa, mu, params, group=None,
                         faces=None, allow_noconv=False):
    """Domain-decomposed CG (FP64 or mixed, as params say) with this rank's
    domain (rank = domain index) in a torch.distributed job; NCCL moves the
    CUDA face buffers."""
    if faces is None:
        faces = domain_faces(slabs, lqcd.LQCD_F64)
    comm = DistributedComm(slabs, rank, faces, group)
    return lqcd.lqcd_dd_cg_solve(ctx, [gauge], [b], [x], [faces], rank, slabs.nt, kappa, mu, params,
                                 antiperiodic_t=slabs.antiperiodic_t, exchange=comm.exchange,
                                 allreduce=comm.allreduce, allow_noconv=allow_noconv, nz=slabs.nz)
