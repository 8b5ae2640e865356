"""Host-side schedule of the slab decomposition (paper_2304_06437_gb300.slabs)
on the CPU: gloo ranks, world sizes 2 and 3, no GPU.

The device half -- which shell records a message carries and where they land
-- is checked on the GPU (tests/test_slabs_gpu.py: every slab bit for bit equal
to the single domain).  Here the transport and its order are checked with a
stand-in slab: a one-dimensional domain of two populations that move one node
up and one node down per step along the slowest axis, with one ghost value
per link face.  Its messages carry (rank, face, step) tags, so every delivery
can be traced, and after k steps the gathered slabs must equal the global
domain shifted k nodes each way -- which holds only if every message reaches
the right neighbour's right ghost before that neighbour's step.
"""
import os
import sys

import numpy as np
import pytest

from paper_2304_06437_gb300 import slabs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_counts_offsets_and_faces():
    assert slabs.slab_counts(10, 3) == [4, 3, 3]
    assert sum(slabs.slab_counts(1031, 8)) == 1031
    assert [slabs.slab_offset(10, 3, r) for r in range(3)] == [0, 4, 7]
    with pytest.raises(ValueError):
        slabs.slab_counts(2, 3)
    L = slabs.LINK
    walls = [1, 1, 1, 2, 1, 1]
    assert slabs.rank_faces(walls, 2, 0, 2) == [1, 1, 1, 2, 1, L]
    assert slabs.rank_faces(walls, 2, 1, 2) == [1, 1, 1, 2, L, 1]
    assert slabs.rank_faces(walls, 2, 0, 1) == walls
    per = [0] * 6
    assert slabs.rank_faces(per, 2, 0, 1) == [0, 0, 0, 0, L, L]
    # 2D: the slowest axis is y
    assert slabs.rank_faces([1, 1, 1, 1, 0, 0], 1, 1, 3) == [1, 1, L, L, 0, 0]
    assert slabs.neighbours(0, 3, True) == (2, 1)
    assert slabs.neighbours(0, 3, False) == (None, 1)
    assert slabs.neighbours(2, 3, False) == (1, None)
    assert slabs.neighbours(0, 1, True) == (0, 0)


class ShiftSlab:
    """Stand-in slab: populations up[i] (moving +1) and dn[i] (moving -1)
    on this rank's nodes; a message is (tag, boundary value)."""

    def __init__(self, rank, up, dn, periodic, world):
        self.rank = rank
        self.up, self.dn = up.astype(np.float64), dn.astype(np.float64)
        self.lo, self.hi = slabs.neighbours(rank, world, periodic)
        self.ghost = {0: None, 1: None}
        self.t = 0
        self.log = []

    def halo_bytes(self):
        return 32  # four float64 values

    def halo_pack(self, side, buf):
        import torch
        # leaving through the low face: the down-mover of node 0; high face:
        # the up-mover of the last node
        v = self.dn[0] if side == 0 else self.up[-1]
        buf.view(torch.float64)[:] = torch.tensor([self.rank, side, self.t, v], dtype=torch.float64)

    def halo_unpack(self, side, buf):
        import torch
        rank, sside, st, v = buf.view(torch.float64).tolist()
        self.log.append((self.t, side, int(rank), int(sside), int(st)))
        self.ghost[side] = v

    def step(self, n):
        assert n == 1
        new_up = np.empty_like(self.up)
        new_dn = np.empty_like(self.dn)
        new_up[1:] = self.up[:-1]
        new_dn[:-1] = self.dn[1:]
        # a wall reflects (halfway bounce-back); a link face takes the ghost
        new_up[0] = self.ghost[0] if self.lo is not None else self.dn[0]
        new_dn[-1] = self.ghost[1] if self.hi is not None else self.up[-1]
        self.up, self.dn = new_up, new_dn
        self.ghost = {0: None, 1: None}
        self.t += 1


def _global(up, dn, steps, periodic):
    up, dn = up.copy(), dn.copy()
    for _ in range(steps):
        nu, nd = np.empty_like(up), np.empty_like(dn)
        nu[1:], nd[:-1] = up[:-1], dn[1:]
        if periodic:
            nu[0], nd[-1] = up[-1], dn[0]
        else:
            nu[0], nd[-1] = dn[0], up[-1]
        up, dn = nu, nd
    return up, dn


def _worker(rank, world, port, periodic, steps, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2304_06437_gb300 import slabs as S
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 11
        g = np.random.Generator(np.random.PCG64(5))
        up, dn = g.random(n), g.random(n)
        counts = S.slab_counts(n, world)
        o = S.slab_offset(n, world, rank)
        slab = ShiftSlab(rank, up[o:o + counts[rank]], dn[o:o + counts[rank]], periodic, world)
        ex = S.HaloExchange(slab, rank, world, periodic, torch)
        ex.step(steps)
        q.put((rank, slab.up.tolist(), slab.dn.tolist(), slab.log))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,periodic", [(2, True), (2, False), (3, True), (3, False)])
def test_exchange_schedule_over_gloo(world, periodic):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() + 17 * world + (1 if periodic else 0)) % 400
    steps = 7
    procs = [ctx.Process(target=_worker, args=(r, world, port, periodic, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every delivery: the low ghost holds the low neighbour's high face, the
    # high ghost the high neighbour's low face, both from the same step
    for rank, _, _, log in out:
        lo, hi = slabs.neighbours(rank, world, periodic)
        want = sorted([(t, 0, lo, 1, t) for t in range(steps) if lo is not None] +
                      [(t, 1, hi, 0, t) for t in range(steps) if hi is not None])
        assert sorted(log) == want, (rank, log)
    # the gathered slabs equal the global domain
    n = 11
    g = np.random.Generator(np.random.PCG64(5))
    up, dn = g.random(n), g.random(n)
    ref_up, ref_dn = _global(up, dn, steps, periodic)
    got_up = np.concatenate([np.array(o[1]) for o in out])
    got_dn = np.concatenate([np.array(o[2]) for o in out])
    assert np.array_equal(got_up, ref_up) and np.array_equal(got_dn, ref_dn)


def test_single_rank_on_a_periodic_axis_links_to_itself():
    import torch
    n = 6
    up, dn = np.arange(n, dtype=float), 10 + np.arange(n, dtype=float)
    slab = ShiftSlab(0, up, dn, True, 1)
    ex = slabs.HaloExchange(slab, 0, 1, True, torch)
    ex.step(4)
    ref_up, ref_dn = _global(up, dn, 4, True)
    assert np.array_equal(slab.up, ref_up) and np.array_equal(slab.dn, ref_dn)
