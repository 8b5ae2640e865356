"""The brick-shape autotuner (lb_autotune).

Every compiled shape of the lattice and storage is timed on a proxy domain and
the fastest is applied.  Shapes only change the schedule, never the per-node
arithmetic, so a tuned domain must step to exactly the bits of an untuned
one; a second domain of the same kind takes the cached choice without timing.
"""
import numpy as np
import pytest

from lbcase import faces_for, random_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import torch
    assert torch.cuda.is_available()
    from paper_2304_06437_gb300 import build
    build.build()
    import paper_2304_06437_gb300 as P
    return P


@pytest.mark.parametrize("lat,dims,storage", [("D3Q19", (70, 24, 30), "f32"), ("D2Q9", (300, 97, 1), "f32"),
                                              ("D3Q27", (40, 26, 20), "f16s")])
def test_autotune_picks_fastest_and_keeps_bits(lb, lat, dims, storage):
    faces, wall_u = faces_for(lat, "lid")
    f0 = np.ascontiguousarray(random_state(lat, dims, 41))
    ref = lb.Solver(lat, dims, 0.6, faces=faces, wall_u=wall_u, storage=storage)
    ref.set_populations(f0)
    ref.step(6)
    want = ref.get_populations()
    ref.close()

    s = lb.Solver(lat, dims, 0.6, faces=faces, wall_u=wall_u, storage=storage)
    s.set_populations(f0)
    s.step(2)  # tuning mid-run: the shell is rebuilt from the current state
    table = s.autotune(steps=3)
    assert len(table) >= 2 and all(e["status"] == 0 for e in table)
    best = min(table, key=lambda e: e["ns_per_update"])
    info = s.info()
    assert (info["tile"][0], info["tile"][1], info["nodes_per_thread"], info["tma_slots"]) == (
        best["bx"], best["by"], best["nodes_per_thread"], best["slots"])
    s.step(4)
    assert np.array_equal(s.get_populations(), want)

    # a second domain of the same kind: cached choice, nothing timed
    s2 = lb.Solver(lat, dims, 0.6, faces=faces, wall_u=wall_u, storage=storage)
    assert s2.autotune(steps=3) == []
    assert s2.info()["tile"][:2] == info["tile"][:2]
    s2.close()
    s.close()
