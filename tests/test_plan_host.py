"""Host logic of the fused scheme's brick planner (lb_plan_fused: the
decomposition lb_create() would choose), on the CPU without a device.

Checked against what the scheme fixes: the bricks tile every grid exactly
once; a sweep is long enough to amortise its pipeline unless the grid is
shallow; the CTA's shared memory fits the 227 KB of an sm_103a CTA; the shell
holds, for every brick face, the outgoing populations of its boundary nodes
(5 per face node for D3Q19, 9 for D3Q27, 3 for D2Q9 -- the directions with a
positive component along an axis); and the benchmark configurations get the
bricks their measurements were taken with.
"""
import itertools

import numpy as np
import pytest

SMEM_MAX = 227 * 1024
OUT_PER_FACE = {"D2Q9": (3, 3), "D3Q19": (5, 5, 5), "D3Q27": (9, 9, 9)}


@pytest.fixture(scope="module")
def P():
    from paper_2304_06437_gb300 import build
    build.build()
    import paper_2304_06437_gb300 as P
    return P


def _internal(lat, dims):
    """(nx, ny, nz) of the library's internal axes: 2D (x, y) -> (x, 1, y)."""
    return (dims[0], 1, dims[1]) if lat == "D2Q9" else tuple(dims)


def _check(lat, dims, p, sms=152):
    nx, ny, nz = _internal(lat, dims)
    # the bricks tile the grid once: the last brick of each axis is the only
    # ragged one
    for n, b, nb in ((nx, p["bx"], p["nbx"]), (ny, p["by"], p["nby"]), (nz, p["bz"], p["nbz"])):
        assert nb * b >= n > (nb - 1) * b, (lat, dims, p)
    assert p["bricks"] == p["nbx"] * p["nby"] * p["nbz"]
    assert 0 < p["shared_bytes"] <= SMEM_MAX
    assert p["tma_slots"] >= 2
    # a sweep amortises its pipeline fill unless the column is shallow
    assert p["bz"] >= min(nz, 8)
    # shell: both sides of every brick face, the outgoing populations of each
    # boundary node
    fx, *rest = OUT_PER_FACE[lat]
    if lat == "D2Q9":
        fy, fz = 0, rest[0]
    else:
        fy, fz = rest
    expect = 2 * (p["nbx"] * fx * ny * nz + p["nby"] * fy * nx * nz + p["nbz"] * fz * nx * ny)
    assert p["shell_elems_per_parity"] == expect, (lat, dims, p, expect)


@pytest.mark.parametrize("lat,dims,storage,tile", [
    ("D3Q19", (1024, 1024, 1024), "f32", (64, 8, 512)),
    ("D3Q19", (1024, 1024, 1024), "f16s", (64, 8, 512)),
    ("D3Q27", (512, 512, 512), "f32", (32, 14, 512)),
    ("D2Q9", (16384, 16384), "f32", (256, 1, 863)),
])
def test_benchmark_configurations_get_their_measured_bricks(P, lat, dims, storage, tile):
    p = P.fused_plan(lat, dims, storage, sms=152)
    assert (p["bx"], p["by"], p["bz"]) == tile
    _check(lat, dims, p)


def test_default_cavity_fills_whole_waves(P):
    """1024^3 D3Q19 on 152 SMs: 2 x 2048 columns = 4096 bricks, 26.95 waves
    of one CTA per SM; the last wave is 95 % full."""
    p = P.fused_plan("D3Q19", (1024, 1024, 1024), sms=152)
    waves = p["bricks"] / 152
    assert p["bricks"] == 4096 and waves / np.ceil(waves) > 0.95


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19", "D3Q27"])
@pytest.mark.parametrize("storage", ["f64", "f32", "f16s", "bf16s"])
def test_bricks_tile_ragged_and_tiny_grids(P, lat, storage):
    rng = np.random.default_rng(7)
    sizes = [1, 2, 3, 7, 31, 33, 64, 65, 127, 129, 300, 1000]
    grids = [(1, 1, 1), (1, 1), (65, 9, 3), (300, 37, 1)]
    for _ in range(12):
        grids.append(tuple(int(v) for v in rng.choice(sizes, 3)))
    for g in grids:
        dims = g[:2] if lat == "D2Q9" else (list(g) + [1, 1])[:3]
        for sms in (152, 148, 1):
            _check(lat, dims, P.fused_plan(lat, dims, storage, sms=sms), sms)


def test_tile_requests_and_rejections(P):
    p = P.fused_plan("D3Q19", (256, 256, 256), "f32", tile=(32, 8, 0), sms=152)
    assert (p["bx"], p["by"]) == (32, 8)
    p = P.fused_plan("D3Q19", (256, 256, 256), "f32", tile=(64, 8, 40), sms=152)
    assert (p["bx"], p["by"], p["bz"], p["nbz"]) == (64, 8, 40, 7)
    from paper_2304_06437_gb300 import LBError
    with pytest.raises(LBError):  # no compiled 48 x 8 brick
        P.fused_plan("D3Q19", (256, 256, 256), "f32", tile=(48, 8, 0))
    for bad in (dict(dims=(0, 4, 4)), dict(dims=(4, 4, 2), lat="D2Q9"), dict(storage=99)):
        args = dict(lat="D3Q19", dims=(8, 8, 8), storage="f32")
        args.update(bad)
        with pytest.raises((LBError, KeyError)):
            P.fused_plan(args["lat"], args["dims"], args["storage"])


def test_pipeline_request_selects_export_warp_variants(P, monkeypatch):
    """The export-warp field of LB_FUSED_PIPELINE picks among the compiled
    alternatives of a brick: 2 decoupled warps, 2 warps inside the per-plane
    barrier (-2), or none (node warps export); -1 takes the shape's default."""
    cases = [("D3Q27", "f32", (32, 14, 0), "2,2,-2", -2), ("D3Q27", "f32", (32, 14, 0), "2,2,-1", -2),
             ("D3Q27", "f32", (32, 14, 0), "2,2,0", 0),
             ("D3Q27", "f32", (32, 10, 0), "2,2,2", 2), ("D3Q19", "f16s", (64, 7, 0), "4,2,-2", -2),
             ("D3Q19", "f16s", (64, 7, 0), "4,2,2", 2), ("D3Q19", "f32", (32, 14, 0), "3,2,-2", -2)]
    for lat, storage, tile, req, want in cases:
        monkeypatch.setenv("LB_FUSED_PIPELINE", req)
        p = P.fused_plan(lat, (256, 256, 256), storage, tile=tile, sms=152)
        assert p["export_warps"] == want and (p["bx"], p["by"]) == tile[:2], (lat, req, p)
        _check(lat, (256, 256, 256), p)
    monkeypatch.delenv("LB_FUSED_PIPELINE")
    assert P.fused_plan("D3Q27", (256, 256, 256), "f32", tile=(32, 14, 0), sms=152)["export_warps"] == -2
    assert P.fused_plan("D3Q19", (256, 256, 256), "f32", sms=152)["export_warps"] == 0
