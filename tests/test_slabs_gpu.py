"""Slab decomposition on the GPU: ranks as contexts on one device.

A domain cut into slabs along its slowest axis (z in 3D, y in 2D), each slab
a context whose faces on that axis are links, with the halo messages moved
between steps (lb_group_*), must compute the single domain's populations bit
for bit: the records a slab reads across a link face are the neighbour's
rounded state collided once more, exactly what a brick face inside one
context carries.  Slab heights are chosen not to be multiples of the sweep
length, so rank boundaries fall inside what would be one brick of the single
domain.  The raw halo calls are also driven by hand through torch buffers
(the path a multi-process run takes with NCCL in between), and a message
packed for the wrong face is refused.
"""
import ctypes

import numpy as np
import pytest

from lbcase import dim_of, faces_for, random_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import torch
    assert torch.cuda.is_available()
    from paper_2304_06437_gb300 import build
    build.build()
    import paper_2304_06437_gb300 as P
    return P


def _dims(lat):
    return (300, 23, 1) if dim_of(lat) == 2 else (37, 21, 23)


def _single(lb, lat, dims, faces, wall_u, storage, force, f0, steps, tile, moments=False):
    with lb.Solver(lat, dims, 0.61, faces=faces, wall_u=wall_u, storage=storage, force=force, tile=tile) as s:
        s.set_populations(np.ascontiguousarray(f0))
        s.step(steps)
        if moments:
            return (s.get_populations(),) + s.moments()
        return s.get_populations()


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19", "D3Q27"])
@pytest.mark.parametrize("fname", ["periodic", "walls", "lid", "duct"])
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_two_slabs_equal_the_single_domain_bitwise(lb, lat, fname, storage):
    dims = _dims(lat)
    faces, wall_u = faces_for(lat, fname)
    force = (2e-5, 1e-5, 0.0) if fname == "duct" else (0.0, 0.0, 0.0)
    f0 = random_state(lat, dims, 71)
    steps = 7
    tile = (0, 0, 5)
    ref = _single(lb, lat, dims, faces, wall_u, storage, force, f0, steps, tile)
    with lb.SlabGroup(lat, dims, 0.61, nranks=2, counts=[9, 14], faces=faces, wall_u=wall_u, storage=storage,
                      force=force, tile=tile) as g:
        g.set_populations(f0)
        g.step(steps)
        g.sync()
        got = g.get_populations()
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("lat,fname,storage,nranks,counts", [
    ("D3Q19", "lid", "f32", 3, [7, 8, 8]),
    ("D3Q19", "periodic", "f32", 3, [5, 12, 6]),
    ("D3Q27", "lid_periodic_z", "f32", 4, [6, 6, 5, 6]),
    ("D2Q9", "lid_periodic_z", "f32", 3, None),
    ("D3Q19", "lid", "f16s", 2, [11, 12]),
    ("D3Q19", "periodic", "bf16s", 2, [12, 11]),
    ("D3Q19", "periodic", "f32", 1, None),
    ("D2Q9", "periodic", "f64", 1, None),
])
def test_slab_groups_equal_the_single_domain_bitwise(lb, lat, fname, storage, nranks, counts):
    dims = _dims(lat)
    faces, wall_u = faces_for(lat, fname)
    f0 = random_state(lat, dims, 72)
    if storage in ("f16s", "bf16s"):
        from oracle.storage import round_populations
        import oracle
        f0 = round_populations(f0, oracle.lattice_tables(lat)[1], storage)
    steps = 6
    ref, r_ref, u_ref = _single(lb, lat, dims, faces, wall_u, storage, (0, 0, 0), f0, steps, None, moments=True)
    with lb.SlabGroup(lat, dims, 0.61, nranks=nranks, counts=counts, faces=faces, wall_u=wall_u,
                      storage=storage) as g:
        g.set_populations(f0)
        g.step(2)
        g.step(steps - 2)
        g.sync()
        got = g.get_populations()
        rho, u = g.moments()
    assert np.array_equal(got, ref)
    assert np.array_equal(rho, r_ref) and np.array_equal(u, u_ref)


def test_halo_calls_by_hand_and_a_mismatched_message(lb):
    """Two linked contexts stepped by hand: pack into torch buffers, unpack on
    the neighbour, one step each -- the schedule of a multi-process run."""
    import torch
    B = lb._binding
    lat, storage = "D3Q19", "f32"
    dims = (29, 17, 19)
    faces, wall_u = faces_for(lat, "lid")
    f0 = random_state(lat, dims, 73)
    ref = _single(lb, lat, dims, faces, wall_u, storage, (0, 0, 0), f0, 5, None)
    nz = [8, 11]
    plane = dims[0] * dims[1]
    parts = []
    for r in range(2):
        fr = list(faces)
        fr[4 + (1 - r)] = B.LB_LINK  # rank 0: +z link; rank 1: -z link
        s = lb.Solver(lat, (dims[0], dims[1], nz[r]), 0.61, faces=fr, wall_u=wall_u, storage=storage,
                      tile=(64, 8, 0))
        n0 = (0 if r == 0 else nz[0]) * plane
        s.set_populations(np.ascontiguousarray(f0[:, n0:n0 + nz[r] * plane]))
        parts.append(s)
    nbytes = parts[0].halo_bytes()
    assert nbytes == parts[1].halo_bytes() and nbytes % 16 == 0  # back-to-back messages stay aligned
    msg = [torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(2)]
    for _ in range(5):
        parts[0].halo_pack(1, msg[0])
        parts[1].halo_pack(0, msg[1])
        for s in parts:
            s.sync()
        parts[0].halo_unpack(1, msg[1])
        parts[1].halo_unpack(0, msg[0])
        for s in parts:
            s.step(1)
    got = np.concatenate([s.get_populations() for s in parts], axis=1)
    assert np.array_equal(got, ref)
    # a linked context takes one step per exchange
    with pytest.raises(lb.LBError):
        parts[0].step(2)
    # a face that is not a link has no halo
    with pytest.raises(lb.LBError):
        parts[0].halo_pack(0, msg[0])
    # a message packed for the same face (rank 0's own high face, not a low
    # face) is refused by the unpack kernel, which records LB_E_INVAL for the
    # next sync and copies nothing
    parts[0].halo_pack(1, msg[0])
    parts[0].sync()
    before = parts[0].get_populations()
    parts[0].halo_unpack(1, msg[0])
    with pytest.raises(lb.LBError) as e:
        parts[0].sync()
    assert e.value.code == B.LB_E_INVAL
    assert np.array_equal(parts[0].get_populations(), before)
    # the status is sticky until the state is set from outside
    with pytest.raises(lb.LBError):
        parts[0].sync()
    parts[0].set_populations(before)
    parts[0].sync()
    for s in parts:
        s.close()
