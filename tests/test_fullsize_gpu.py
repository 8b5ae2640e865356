"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (fused scheme, FP32 storage, the library's default brick shape).

The oracle cannot step a 1024^3 grid, so these tests sample: a few small
boxes of the GPU state are read at step t and t + 1; the oracle advances each
box one step in FP64 and the two are compared node by node.  A box face that
is a real domain face keeps its kind (wall or moving lid); any other box face
is cut out of the grid, so the oracle treats it as a wall and the layer of
nodes next to it (whose upstream neighbours lie outside the box) is left out
of the comparison.  Boxes are placed on the domain corners, on the lid, across
the brick boundaries of the launch (where the shell exchange carries the
populations) and, on periodic axes, across the periodic wrap.
"""
import numpy as np
import pytest

import oracle
import synth
from lbcase import faces_for, rel_l2
from oracle.storage import quantum

pytestmark = pytest.mark.gpu

BOX = 6
FTOL_F32 = 2e-6  # one FP32 step of populations of size ~0.3


@pytest.fixture(scope="module")
def Solver():
    import torch
    assert torch.cuda.is_available()
    from paper_2304_06437_gb300 import build
    build.build()
    from paper_2304_06437_gb300 import Solver as S
    return S


def _segments(lo, size, n):
    """Contiguous pieces (start, length, offset in the box) of a possibly
    wrapped range [lo, lo + size) on an axis of length n."""
    lo %= n
    if lo + size <= n:
        return [(lo, size, 0)]
    first = n - lo
    return [(lo, first, 0), (0, size - first, first)]


def read_box(s, lo, size):
    """Populations [q][size_z][size_y][size_x] of a box that may wrap around
    periodic axes (read as up to eight plain regions)."""
    nx, ny, nz = s.dims
    out = np.empty((s.q, size[2], size[1], size[0]))
    for xs, xl, xo in _segments(lo[0], size[0], nx):
        for ys, yl, yo in _segments(lo[1], size[1], ny):
            for zs, zl, zo in _segments(lo[2], size[2], nz):
                part = s.get_region((xs, ys, zs), (xl, yl, zl)).reshape(s.q, zl, yl, xl)
                out[:, zo:zo + zl, yo:yo + yl, xo:xo + xl] = part
    return out


def box_case(lat, dims, faces, wall_u, lo, size):
    """Oracle configuration of a box and the mask of nodes it can predict."""
    box_faces, box_wall = [], []
    keep = np.ones((size[2], size[1], size[0]), dtype=bool)
    for ax in range(3):
        n = dims[ax]
        for side in (0, 1):
            k = 2 * ax + side
            if size[ax] == n and faces[k] == 0 and lo[ax] == 0:
                box_faces.append(0)  # the whole periodic axis is in the box
                box_wall.append([0, 0, 0])
                continue
            on_face = (lo[ax] == 0) if side == 0 else (lo[ax] + size[ax] == n)
            if faces[k] != 0 and on_face:
                box_faces.append(faces[k])
                box_wall.append(list(wall_u[k]) if wall_u is not None else [0, 0, 0])
            else:
                box_faces.append(1)  # cut face: the adjacent layer is not comparable
                box_wall.append([0, 0, 0])
                sl = [slice(None)] * 3
                sl[2 - ax] = 0 if side == 0 else size[ax] - 1
                keep[tuple(sl)] = False
    return box_faces, box_wall, keep


def boxes_for(s, dims, faces, seed):
    """Corners, lid, brick junctions (of the launch's brick shape), wrap and
    random interior boxes."""
    bx, by, bz = s.info()["tile"]
    nx, ny, nz = dims
    d3 = nz > 1
    size = (BOX, BOX, BOX if d3 else 1)
    out = []
    for cx in (0, nx - BOX):
        for cy in (0, ny - BOX):
            for cz in ((0, nz - BOX) if d3 else (0,)):
                out.append((cx, cy, cz))
    out.append((nx // 2 - 3, ny - BOX, nz // 2 - 3 if d3 else 0))  # lid centre (or top edge)
    # junctions of bricks (x, y, z boundaries of the brick grid; 2D: x and the sweep axis)
    jx = min(nx - BOX, max(0, (nx // bx // 2) * bx - 3))
    if d3:
        jy = min(ny - BOX, max(0, (ny // by // 2) * by - 3))
        jz = min(nz - BOX, max(0, bz - 3))
    else:
        jy = min(ny - BOX, max(0, bz - 3))  # 2D grids sweep along y
        jz = 0
    out.append((jx, jy, jz))
    out.append((bx - 3, by - 3 if d3 else jy, jz))
    if faces[0] == 0:  # wrap on periodic axes
        out.append((nx - 3, ny - 3 if faces[2] == 0 else ny // 3, (nz - 3 if faces[4] == 0 else nz // 3) if d3 else 0))
    g = synth.rng(seed)
    for _ in range(2):
        out.append((int(g.integers(0, nx - BOX)), int(g.integers(0, ny - BOX)),
                    int(g.integers(0, nz - BOX)) if d3 else 0))
    return out, size


def check_sampled(Solver, lat, dims, tau, fname, init, warm_steps, seed, storage="f32"):
    import torch
    faces, wall_u = faces_for(lat, fname)
    s = Solver(lat, dims, tau, faces=faces, wall_u=wall_u, storage=storage)
    init(s, torch)
    s.step(warm_steps)
    s.sync()
    boxes, size = boxes_for(s, s.dims, faces, seed)
    before = [read_box(s, lo, size) for lo in boxes]
    s.step(1)
    s.sync()
    after = [read_box(s, lo, size) for lo in boxes]
    s.close()
    worst = 0.0
    for lo, f0, f1 in zip(boxes, before, after):
        bf, bw, keep = box_case(lat, s.dims, faces, wall_u, lo, size)
        cfg = oracle.make_cfg(lat, size, tau, faces=bf, wall_u=bw)
        got = f1.reshape(s.q, -1)
        k = keep.reshape(-1)
        assert k.sum() > 0
        if storage == "f32":
            ref = oracle.run(cfg, np.ascontiguousarray(f0.reshape(s.q, -1)), 1)
            err = np.abs(got[:, k] - ref[:, k]).max()
            assert err < FTOL_F32, (lo, err)
        else:
            # reduced storage: the oracle step rounded to the format, within
            # one unit of the format (plus FP32 resolution near zero)
            ref = oracle.run_stored(cfg, np.ascontiguousarray(f0.reshape(s.q, -1)), 1, storage)
            w = oracle.lattice_tables(lat)[1][:, None]
            dg, dr = got - w, ref - w
            ulp = np.maximum(quantum(dg, storage), quantum(dr, storage))
            err = (np.abs(dg - dr) / (ulp + 1e-7))[:, k].max()
            assert err <= 1.0 + 1e-9, (lo, err)
        worst = max(worst, err)
        r_ref, u_ref = oracle.moments(cfg, ref)
        r_got, u_got = oracle.moments(cfg, np.ascontiguousarray(got))
        tol = 1e-5 if storage == "f32" else 1e-2
        assert rel_l2(r_got[k], r_ref[k]) < tol
        assert rel_l2(u_got[:, k], u_ref[:, k]) < tol, (lo, rel_l2(u_got[:, k], u_ref[:, k]))
    return worst


def _tg3d(n, u0, tau):
    def init(s, torch):
        rho, u, _ = synth.taylor_green_3d_torch(n, u0, 1.0, tau, torch, pineq=False)
        s.init_moments(rho, u)
        del rho, u
        torch.cuda.empty_cache()
    return init


def test_cavity_d3q19_1024_sampled(Solver):
    """D3Q19 lid-driven cavity, 1024^3, FP32, tau 0.52, lid 0.05: a smooth
    vortex field is set inside the walled box so every sampled node moves."""
    check_sampled(Solver, "D3Q19", (1024, 1024, 1024), 0.52, "lid", _tg3d(1024, 0.02, 0.52), 3, 11)


def test_cavity_d3q19_1024_f16s_sampled(Solver):
    """The same cavity with shifted FP16 storage (bench.py --storage f16s):
    one step within one storage unit of the rounded oracle step."""
    check_sampled(Solver, "D3Q19", (1024, 1024, 1024), 0.52, "lid", _tg3d(1024, 0.02, 0.52), 3, 21, "f16s")


def test_tg_d3q27_512_bf16s_sampled(Solver):
    """D3Q27 512^3 Taylor-Green with shifted BF16 storage."""
    def init(s, torch):
        rho, u, pi = synth.taylor_green_3d_torch(512, 0.02, 1.0, 0.8, torch)
        s.init_moments(rho, u, pi)
    check_sampled(Solver, "D3Q27", (512, 512, 512), 0.8, "periodic", init, 3, 22, "bf16s")


def test_tg_d3q27_512_sampled(Solver):
    """D3Q27 periodic Taylor-Green, 512^3, FP32, u0 0.02, tau 0.8."""
    def init(s, torch):
        rho, u, pi = synth.taylor_green_3d_torch(512, 0.02, 1.0, 0.8, torch)
        s.init_moments(rho, u, pi)
    check_sampled(Solver, "D3Q27", (512, 512, 512), 0.8, "periodic", init, 3, 12)


def test_tg_d2q9_16384_sampled(Solver):
    """D2Q9 periodic Taylor-Green, 16384^2, FP32, u0 0.01, tau 0.8."""
    def init(s, torch):
        rho, u, pi = synth.taylor_green_2d_torch(16384, 0.01, 1.0, 0.8, torch)
        s.init_moments(rho, u, pi)
    check_sampled(Solver, "D2Q9", (16384, 16384), 0.8, "periodic", init, 3, 13)


def test_tg_d3q27_1024_sampled(Solver):
    """D3Q27 periodic Taylor-Green at 1.07e9 nodes (bench.py --workload
    tg_d3q27_1024: FP32, 116 GB of populations, 32 x 14 bricks)."""
    def init(s, torch):
        rho, u, pi = synth.taylor_green_3d_torch(1024, 0.02, 1.0, 0.8, torch)
        s.init_moments(rho, u, pi)
        del rho, u, pi
        torch.cuda.empty_cache()
    check_sampled(Solver, "D3Q27", (1024, 1024, 1024), 0.8, "periodic", init, 3, 14)


def test_tg_d3q27_1024_f16s_sampled(Solver):
    """The same with shifted FP16 storage (32 x 16 bricks)."""
    def init(s, torch):
        rho, u, pi = synth.taylor_green_3d_torch(1024, 0.02, 1.0, 0.8, torch)
        s.init_moments(rho, u, pi)
        del rho, u, pi
        torch.cuda.empty_cache()
    check_sampled(Solver, "D3Q27", (1024, 1024, 1024), 0.8, "periodic", init, 3, 24, "f16s")
