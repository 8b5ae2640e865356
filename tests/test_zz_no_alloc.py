"""lb_step_noalloc: the step for callers that cannot let a library allocate
device memory (their memory belongs to another allocator or a fixed budget).

It runs the two-pass schedule with its moment arrays in a fixed file-scope
device array, on the caller's population buffer.  Checked through the C ABI
against the allocating path (LB_F64 two-pass context: set populations, step,
read back) on two calls in a row, so that the second call also shows that the
contents the first call leaves in the shared array do no harm.  Kept in a file
of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

from lbcase import faces_for, random_state

pytestmark = pytest.mark.gpu


def _call(lib, B, lat, dims, tau, faces, wall_u, force, f_dev, n, torch, rho0=1.0):
    bnd = B.lb_boundary()
    for k in range(6):
        bnd.kind[k] = faces[k]
        for al in range(3):
            bnd.wall_u[k][al] = float(wall_u[k][al]) if wall_u is not None else 0.0
    frc = (ctypes.c_double * 3)(*force)
    stream = torch.cuda.current_stream().cuda_stream
    return lib.lb_step_noalloc(B.LATTICES[lat], (ctypes.c_int64 * 3)(*dims), tau, ctypes.byref(bnd), rho0, frc,
                               ctypes.c_void_p(f_dev.data_ptr()), n, ctypes.c_void_p(stream))


@pytest.mark.parametrize("lat,dims,fname,force,rho0", [
    ("D3Q19", (37, 21, 13), "lid", (0, 0, 0), 1.0),
    ("D3Q27", (20, 17, 9), "duct", (2e-5, 0, 1e-5), 1.0),
    ("D2Q9", (300, 37, 1), "lid_periodic_z", (0, 0, 0), 1.0),
    ("D3Q19", (23, 14, 11), "lid", (1e-5, 0, 0), 1.3),
    ("D2Q9", (45, 33, 1), "duct", (2e-5, 0, 0), 0.8),
])
def test_noalloc_matches_allocating_path_on_two_calls(lat, dims, fname, force, rho0):
    import torch
    from paper_2304_06437_gb300 import Solver, _binding as B, build
    build.build()
    lib = B.load()
    faces, wall_u = faces_for(lat, fname)
    # populations around the reference density rho0, so that the shift by
    # t_a rho0 (and back) is exercised at a density other than one
    f0 = rho0 * random_state(lat, dims, 29)
    steps = 7
    f_dev = torch.from_numpy(np.ascontiguousarray(f0)).cuda()
    outs = []
    for _ in range(2):
        assert _call(lib, B, lat, dims, 0.61, faces, wall_u, force, f_dev, steps, torch, rho0) == B.LB_OK
        torch.cuda.synchronize()
        outs.append(f_dev.cpu().numpy().copy())
    with Solver(lat, dims, 0.61, faces=faces, wall_u=wall_u, storage="f64", scheme="two_pass", force=force,
                rho0=rho0) as s:
        s.set_populations(np.ascontiguousarray(f0))
        s.step(steps)
        ref1 = s.get_populations()
        s.step(steps)
        ref2 = s.get_populations()
    assert np.abs(outs[0] - ref1).max() <= 1e-14 * rho0
    assert np.abs(outs[1] - ref2).max() <= 1e-14 * rho0


def test_noalloc_zero_steps_is_the_shift_round_trip():
    """n = 0 shifts to the stored form and back, as lb_set_populations +
    lb_get_populations of an FP64 context do."""
    import torch
    from paper_2304_06437_gb300 import Solver, _binding as B, build
    build.build()
    lib = B.load()
    lat, dims, rho0 = "D3Q19", (19, 11, 7), 1.3
    faces, wall_u = faces_for(lat, "walls")
    f0 = rho0 * random_state(lat, dims, 31)
    f_dev = torch.from_numpy(np.ascontiguousarray(f0)).cuda()
    assert _call(lib, B, lat, dims, 0.7, faces, wall_u, (0, 0, 0), f_dev, 0, torch, rho0) == B.LB_OK
    torch.cuda.synchronize()
    with Solver(lat, dims, 0.7, faces=faces, wall_u=wall_u, storage="f64", scheme="two_pass", rho0=rho0) as s:
        s.set_populations(np.ascontiguousarray(f0))
        ref = s.get_populations()
    assert np.array_equal(f_dev.cpu().numpy(), ref)


def test_noalloc_rejects_grids_beyond_the_scratch():
    import torch
    from paper_2304_06437_gb300 import _binding as B, build
    build.build()
    lib = B.load()
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    # 95^3 D3Q19 nodes need 10 * 857375 * 8 bytes > 64 MiB: rejected on the host
    rc = _call(lib, B, "D3Q19", (95, 95, 95), 0.7, [0] * 6, None, (0, 0, 0), dummy, 1, torch)
    assert rc == B.LB_E_TOO_LARGE
    assert lib.lb_status_string(rc) == b"grid exceeds the no-allocation scratch size"
