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


def _call(lib, B, lat, dims, tau, faces, wall_u, force, f_dev, n, torch):
    bnd = B.lb_boundary()
    for k in range(6):
        bnd.kind[k] = faces[k]
        for al in range(3):
            bnd.wall_u[k][al] = float(wall_u[k][al]) if wall_u is not None else 0.0
    frc = (ctypes.c_double * 3)(*force)
    stream = torch.cuda.current_stream().cuda_stream
    return lib.lb_step_noalloc(B.LATTICES[lat], (ctypes.c_int64 * 3)(*dims), tau, ctypes.byref(bnd), 1.0, frc,
                               ctypes.c_void_p(f_dev.data_ptr()), n, ctypes.c_void_p(stream))


@pytest.mark.parametrize("lat,dims,fname,force", [
    ("D3Q19", (37, 21, 13), "lid", (0, 0, 0)),
    ("D3Q27", (20, 17, 9), "duct", (2e-5, 0, 1e-5)),
    ("D2Q9", (300, 37, 1), "lid_periodic_z", (0, 0, 0)),
])
def test_noalloc_matches_allocating_path_on_two_calls(lat, dims, fname, force):
    import torch
    from paper_2304_06437_gb300 import Solver, _binding as B, build
    build.build()
    lib = B.load()
    faces, wall_u = faces_for(lat, fname)
    f0 = random_state(lat, dims, 29)
    steps = 7
    f_dev = torch.from_numpy(np.ascontiguousarray(f0)).cuda()
    outs = []
    for _ in range(2):
        assert _call(lib, B, lat, dims, 0.61, faces, wall_u, force, f_dev, steps, torch) == B.LB_OK
        torch.cuda.synchronize()
        outs.append(f_dev.cpu().numpy().copy())
    with Solver(lat, dims, 0.61, faces=faces, wall_u=wall_u, storage="f64", scheme="two_pass", force=force) as s:
        s.set_populations(np.ascontiguousarray(f0))
        s.step(steps)
        ref1 = s.get_populations()
        s.step(steps)
        ref2 = s.get_populations()
    assert np.abs(outs[0] - ref1).max() <= 1e-14
    assert np.abs(outs[1] - ref2).max() <= 1e-14


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
