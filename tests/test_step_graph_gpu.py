"""lb_step's replay of a captured pair of fused steps (one CUDA graph launch
per two steps for runs of four or more steps): bit for bit the same
populations as stepping one launch at a time, from either shell parity,
after the brick plan changes under it (a batch re-plans its members), and
when the caller is itself capturing the library's stream."""
import numpy as np
import pytest

from lbcase import faces_for, random_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Solver():
    import torch
    assert torch.cuda.is_available()
    from paper_2304_06437_gb300 import build
    build.build()
    from paper_2304_06437_gb300 import Solver as S
    return S


def _plain(Solver, lat, dims, faces, wall_u, storage, f0, total, force=(0, 0, 0)):
    with Solver(lat, dims, 0.6, faces=faces, wall_u=wall_u, storage=storage, force=force) as s:
        s.set_populations(np.ascontiguousarray(f0))
        for _ in range(total):
            s.step(1)
        return s.get_populations()


@pytest.mark.parametrize("lat,storage,fname", [("D3Q19", "f32", "lid"), ("D3Q27", "f32", "duct"),
                                               ("D2Q9", "f16s", "periodic"), ("D3Q19", "f64", "walls")])
def test_graph_runs_equal_single_launches(Solver, lat, storage, fname):
    dims = (300, 37, 1) if lat == "D2Q9" else (37, 21, 13)
    faces, wall_u = faces_for(lat, fname)
    force = (2e-5, 0, 1e-5) if fname == "duct" else (0, 0, 0)
    f0 = random_state(lat, dims, 83)
    # 11 (5 pairs + 1), then 1 + 10 (captured at the other parity), 3 single
    # launches and 6 (one step to re-align the parity, 2 pairs, 1 step)
    with Solver(lat, dims, 0.6, faces=faces, wall_u=wall_u, storage=storage, force=force) as s:
        s.set_populations(np.ascontiguousarray(f0))
        s.step(11)
        got11 = s.get_populations()
    with Solver(lat, dims, 0.6, faces=faces, wall_u=wall_u, storage=storage, force=force) as s:
        s.set_populations(np.ascontiguousarray(f0))
        for n in (1, 10, 3, 6):
            s.step(n)
        got20 = s.get_populations()
        assert s.info()["steps_done"] == 20
    assert np.array_equal(got11, _plain(Solver, lat, dims, faces, wall_u, storage, f0, 11, force))
    assert np.array_equal(got20, _plain(Solver, lat, dims, faces, wall_u, storage, f0, 20, force))


def test_graph_dropped_when_a_batch_replans(Solver):
    from paper_2304_06437_gb300 import Batch
    lat, dims, storage = "D3Q19", (32, 16, 20), "f32"
    faces, wall_u = faces_for(lat, "lid")
    f0 = random_state(lat, dims, 84)
    with Solver(lat, dims, 0.6, faces=faces, wall_u=wall_u, storage=storage) as s:
        s.set_populations(np.ascontiguousarray(f0))
        s.step(8)
        tile0 = s.info()["tile"]
        b = Batch([s])
        b.step(3)
        b.sync()
        b.close()
        tile1 = s.info()["tile"]
        s.step(8)
        got = s.get_populations()
    assert tile1 != tile0  # the batch gave the member one brick per column
    assert np.array_equal(got, _plain(Solver, lat, dims, faces, wall_u, storage, f0, 19))


def test_caller_capture_of_lb_step(Solver):
    """A caller capturing the library's stream records lb_step's launches in
    its own graph (lb_step does not start a capture of its own then)."""
    import torch
    lat, dims, storage = "D3Q19", (37, 21, 13), "f32"
    faces, wall_u = faces_for(lat, "lid")
    f0 = random_state(lat, dims, 85)
    st = torch.cuda.Stream()
    with Solver(lat, dims, 0.6, faces=faces, wall_u=wall_u, storage=storage, stream=st) as s:
        s.set_populations(np.ascontiguousarray(f0))
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            s.step(6)
        for _ in range(2):
            g.replay()
        torch.cuda.synchronize()
        got = s.get_populations()
    assert np.array_equal(got, _plain(Solver, lat, dims, faces, wall_u, storage, f0, 12))
