"""Slab decomposition across processes: one rank per GPU, torch.distributed
as the transport.

Each rank owns a slab of the domain along its slowest axis (z in 3D, y in 2D)
as a Solver whose faces on that axis are LB_LINK where it borders another
rank.  Before every step the populations that leave a slab through a link
face travel to the neighbour as one message (lb_halo_pack on the sender,
lb_halo_unpack on the receiver); the library then takes one launch.  On GPUs
the messages are CUDA tensors sent with NCCL into the receiver's own memory;
no kernel ever reads another GPU's memory.

This module holds the host-side schedule only -- which rank sends which face
to whom, in which order -- so that it can be checked with the gloo backend on
the CPU, with any object that offers halo_bytes / halo_pack / halo_unpack /
step in place of a Solver.
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

LINK = 3  # LB_LINK


def slab_counts(extent: int, world: int) -> List[int]:
    """Planes per rank along the slowest axis: as even as possible, the first
    extent % world ranks one plane thicker (the split lb_group_create makes)."""
    if world < 1 or extent < world:
        raise ValueError("need 1 <= world <= extent")
    return [extent // world + (1 if r < extent % world else 0) for r in range(world)]


def slab_offset(extent: int, world: int, rank: int) -> int:
    return sum(slab_counts(extent, world)[:rank])


def rank_faces(faces: Sequence[int], slow_axis: int, rank: int, world: int) -> List[int]:
    """The face kinds of rank `rank`'s slab: LB_LINK between slabs, and at the
    ends of a periodic slowest axis (the last slab links to the first)."""
    out = [int(k) for k in faces]
    if LINK in out:
        raise ValueError("the global faces may not be links")
    lo, hi = 2 * slow_axis, 2 * slow_axis + 1
    periodic = out[lo] == 0
    if rank > 0 or periodic:
        out[lo] = LINK
    if rank < world - 1 or periodic:
        out[hi] = LINK
    return out


def neighbours(rank: int, world: int, periodic: bool) -> Tuple[Optional[int], Optional[int]]:
    """(low, high) neighbour ranks of a slab; None where the slab ends at a
    wall of the global domain."""
    lo = rank - 1 if rank > 0 else (world - 1 if periodic else None)
    hi = rank + 1 if rank < world - 1 else (0 if periodic else None)
    return lo, hi


class HaloExchange:
    """The per-step exchange of one rank.

    Message order: with two ranks on a periodic axis both neighbours are the
    same rank, and NCCL matches point-to-point messages between two ranks in
    the order they were posted, without tags.  So every rank posts its sends
    high face first, low face second, and its receives low face first, high
    face second: the peer's first message (its high face) lands in this rank's
    low ghost, its second (its low face) in the high ghost -- the pairing the
    ring needs.  A rank that is its own neighbour (one rank, periodic) copies
    locally."""

    def __init__(self, slab, rank: int, world: int, periodic: bool, torch, device=None, group=None):
        self.slab = slab
        self.rank, self.world = rank, world
        self.lo, self.hi = neighbours(rank, world, periodic)
        self.torch = torch
        self.group = group
        n = slab.halo_bytes()
        # messages are bytes, 16-byte aligned (allocations are)
        mk = (lambda: torch.empty(n, dtype=torch.uint8, device=device))
        self.send = {s: mk() for s in (0, 1) if self._nbr(s) is not None}
        self.recv = {s: mk() for s in (0, 1) if self._nbr(s) is not None}

    def _nbr(self, side):
        return self.lo if side == 0 else self.hi

    def exchange(self):
        dist = self.torch.distributed
        for s in self.send:
            self.slab.halo_pack(s, self.send[s])
        self._fence()
        ops = []
        for s in (1, 0):  # sends: high face first
            nb = self._nbr(s)
            if nb is not None and nb != self.rank:
                ops.append(dist.P2POp(dist.isend, self.send[s], nb, group=self.group))
        for s in (0, 1):  # receives: low face first
            nb = self._nbr(s)
            if nb is not None and nb != self.rank:
                ops.append(dist.P2POp(dist.irecv, self.recv[s], nb, group=self.group))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        for s in (0, 1):
            if self._nbr(s) == self.rank:
                # one rank on a periodic axis: its own high face is its low ghost
                self.recv[s].copy_(self.send[1 - s])
        for s in self.recv:
            self.slab.halo_unpack(s, self.recv[s])

    def _fence(self):
        # the packs run on the slab's stream; the transport must see them
        sync = getattr(self.slab, "sync", None)
        if sync is not None:
            sync()

    def step(self, n: int = 1):
        for _ in range(int(n)):
            self.exchange()
            self.slab.step(1)
