"""One lattice split along z into slabs (one per GPU or rank).

Streaming and the force of Eq. (3) reach one plane across a slab's faces (periodic
boundaries with forces computed across them, Sec. II A), so before every step each
slab sends its 2 lowest and 2 highest planes to the 2 ghost planes below and above
its neighbours (periodic in z) and then takes an ordinary fused step; its own planes
then hold exactly what the same planes of one lattice hold (include/sc_lbm.h,
sc_slab_*). After a step the ghost planes of the current buffer hold the slab's own
view of its neighbours' planes, not theirs, and the canonical state of a slab's
boundary planes (read-outs, diagnostics) is formed from its ghosts: so the groups
below exchange again before the state is read (``sync``). This module only
marshals: the library packs and unpacks the planes on the device, torch copies them
between slabs on one GPU or sends them between ranks (torch.distributed, NCCL on
GPUs, gloo on CPU tensors).
"""
from __future__ import annotations

import ctypes as C

from . import Lattice, make_params
from ._native import check, load

GHOSTS = 2


def slab_ranges(nz: int, parts: int):
    """Contiguous plane ranges [z0, z1) covering nz planes with `parts` slabs of
    nearly equal thickness (differing by at most one plane), each at least 2 planes."""
    if parts < 1 or nz < GHOSTS * parts:
        raise ValueError(f"{nz} planes cannot be split into {parts} slabs of at least {GHOSTS} planes")
    return [(k * nz // parts, (k + 1) * nz // parts) for k in range(parts)]


def exchange_ring(send_low, send_high, recv_low, recv_high, rank: int, world: int, dist=None):
    """The ghost exchange of one rank: its low ghosts receive the lower neighbour's
    high planes, its high ghosts the upper neighbour's low planes (neighbours rank - 1
    and rank + 1, periodic). One rank (world == 1) is its own neighbour on both sides."""
    if world == 1:
        recv_low.copy_(send_high)
        recv_high.copy_(send_low)
        return
    lower, upper = (rank - 1) % world, (rank + 1) % world
    # posted in the same order on every rank, so with two ranks (lower == upper) the
    # first message between a pair is the low planes and the second the high planes
    ops = [dist.P2POp(dist.isend, send_low, lower), dist.P2POp(dist.irecv, recv_high, upper),
           dist.P2POp(dist.isend, send_high, upper), dist.P2POp(dist.irecv, recv_low, lower)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()


class Slab(Lattice):
    """Planes [z0, z1) of the lattice described by ``params`` (the same dictionary a
    Lattice takes; two-lattice layout) with 2 ghost planes on each side. Every Lattice
    method applies to the slab's local planes (ghosts included: local plane 2 is plane
    z0); ``own`` selects the own planes of a local array."""

    def __init__(self, params: dict, z0: int, z1: int, device=None, stream=None):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self._p = make_params(params)
        self.params = dict(params)
        self.z0, self.z1 = int(z0), int(z1)
        self.nx, self.ny = self._p.nx, self._p.ny
        self.nz = self.z1 - self.z0 + 2 * GHOSTS
        self.n = self.nx * self.ny * self.nz
        self.shape = (self.nz, self.ny, self.nx)
        with torch.cuda.device(self.device):
            self.stream = stream or torch.cuda.current_stream(self.device)
            h = C.c_void_p()
            check(load().sc_slab_create(C.byref(self._p), self.z0, self.z1, C.c_void_p(self.stream.cuda_stream),
                                        C.byref(h)))
            self._h = h
            face = C.c_size_t()
            check(load().sc_slab_info(self._h, None, None, None, C.byref(face)))
            self.face_bytes = int(face.value)
            mk = lambda: torch.empty(self.face_bytes, dtype=torch.uint8, device=self.device)
            self.send = [mk(), mk()]
            self.recv = [mk(), mk()]

    @property
    def own(self):
        return slice(GHOSTS, self.nz - GHOSTS)

    def pack(self) -> None:
        for side in (0, 1):
            check(load().sc_slab_pack(self._h, side, C.c_void_p(self.send[side].data_ptr())))

    def unpack(self) -> None:
        for side in (0, 1):
            check(load().sc_slab_unpack(self._h, side, C.c_void_p(self.recv[side].data_ptr())))


class LocalSlabs:
    """Several slabs of one lattice on one device, exchanging through device copies on
    the current stream: the single-GPU form of the decomposition."""

    def __init__(self, params: dict, parts: int, device=None):
        self.slabs = [Slab(params, z0, z1, device=device) for z0, z1 in slab_ranges(params["nz"], parts)]
        self.stale = True

    def init(self, init: dict) -> None:
        for s in self.slabs:
            s.init(init)
        self.stale = True

    def exchange(self) -> None:
        n = len(self.slabs)
        for s in self.slabs:
            s.pack()
        for k, s in enumerate(self.slabs):
            s.recv[0].copy_(self.slabs[(k - 1) % n].send[1])
            s.recv[1].copy_(self.slabs[(k + 1) % n].send[0])
        for s in self.slabs:
            s.unpack()

    def step(self, n: int = 1) -> None:
        for _ in range(int(n)):
            self.exchange()
            for s in self.slabs:
                s.step(1)
        self.stale = self.stale or int(n) > 0

    def sync(self) -> None:
        """Exchange the ghost planes once more, so every slab's read-outs and diagnostics
        see its neighbours' current planes."""
        if self.stale:
            self.exchange()
            self.stale = False

    def close(self) -> None:
        for s in self.slabs:
            s.close()


class DistributedSlab:
    """This rank's slab of one lattice split over all ranks of torch.distributed's
    default group (rank r holds slab_ranges(nz, world)[r]); every step exchanges the
    ghost planes with the two neighbouring ranks."""

    def __init__(self, params: dict, device=None):
        import torch.distributed as dist
        self.dist = dist
        self.rank, self.world = dist.get_rank(), dist.get_world_size()
        z0, z1 = slab_ranges(params["nz"], self.world)[self.rank]
        self.slab = Slab(params, z0, z1, device=device)
        self.stale = True

    def init(self, init: dict) -> None:
        self.slab.init(init)
        self.stale = True

    def exchange(self) -> None:
        s = self.slab
        s.pack()
        exchange_ring(s.send[0], s.send[1], s.recv[0], s.recv[1], self.rank, self.world, self.dist)
        s.unpack()

    def step(self, n: int = 1) -> None:
        for _ in range(int(n)):
            self.exchange()
            self.slab.step(1)
        self.stale = self.stale or int(n) > 0

    def sync(self) -> None:
        """Exchange once more before the state is read (every rank must call it)."""
        if self.stale:
            self.exchange()
            self.stale = False

    def close(self) -> None:
        self.slab.close()
