"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (the benchmark spec): relative L2 on rho and u of 1e-12 in FP64 and 1e-5
in FP32 storage/arithmetic; populations are also compared element by element.
The fused single-array schedule must equal the paper's two-pass schedule bit
for bit (same per-node arithmetic, lb_collide.cuh), and must not depend on the
brick shape (a race would make it schedule dependent).
"""
import numpy as np
import pytest

import oracle
import synth
from lbcase import dim_of, faces_for, oracle_cfg, random_state, rel_l2
from oracle.storage import round_populations

pytestmark = pytest.mark.gpu

LATTICES = ["D2Q9", "D3Q19", "D3Q27"]
TOL = {"f64": 1e-12, "f32": 1e-5}
FTOL = {"f64": 1e-14, "f32": 2e-7}


@pytest.fixture(scope="module")
def Solver():
    import torch
    assert torch.cuda.is_available()
    from paper_2304_06437_gb300 import build
    build.build()
    from paper_2304_06437_gb300 import Solver as S
    return S


def _dims(lat, kind="ragged"):
    if dim_of(lat) == 2:
        return {"ragged": (300, 37, 1), "tiny": (7, 5, 1)}[kind]
    return {"ragged": (37, 21, 13), "tiny": (5, 4, 3)}[kind]


def _run_pair(Solver, lat, dims, tau, fname, storage, scheme, steps, force=(0, 0, 0), tile=None, seed=101):
    faces, wall_u = faces_for(lat, fname)
    f0 = random_state(lat, dims, seed)
    cfg = oracle_cfg(lat, dims, tau, faces, wall_u, force=force)
    ref = oracle.run(cfg, f0, steps)
    s = Solver(lat, dims, tau, faces=faces, wall_u=wall_u, storage=storage, scheme=scheme, force=force, tile=tile)
    s.set_populations(np.ascontiguousarray(f0))
    s.step(steps)
    s.sync()
    got = s.get_populations()
    rho, u = s.moments()
    s.close()
    return ref, got, cfg, rho, u


@pytest.mark.parametrize("lat", LATTICES)
@pytest.mark.parametrize("fname", ["periodic", "walls", "lid", "duct", "lid_periodic_z"])
@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("scheme", ["fused", "two_pass"])
def test_one_and_ten_steps_match_oracle(Solver, lat, fname, storage, scheme):
    dims = _dims(lat)
    force = (2e-5, 1e-5, 0.0) if fname == "duct" else (0, 0, 0)
    # a short sweep length so that z-bricks and their shells are exercised
    tile = None if scheme == "two_pass" else (0, 0, 5)
    for steps in (1, 10):
        ref, got, cfg, rho, u = _run_pair(Solver, lat, dims, 0.62, fname, storage, scheme, steps, force=force,
                                          tile=tile)
        assert np.abs(got - ref).max() < FTOL[storage] * 10 * steps, (steps, np.abs(got - ref).max())
        r_ref, u_ref = oracle.moments(cfg, ref)
        assert rel_l2(rho, r_ref) < TOL[storage]
        assert rel_l2(u, u_ref) < TOL[storage], rel_l2(u, u_ref)


@pytest.mark.parametrize("lat", LATTICES)
@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("fname", ["lid", "periodic", "duct"])
def test_fused_equals_two_pass_bitwise(Solver, lat, storage, fname):
    dims = _dims(lat)
    faces, wall_u = faces_for(lat, fname)
    force = (2e-5, 0, 1e-5) if fname == "duct" else (0, 0, 0)
    f0 = random_state(lat, dims, 7)
    outs = []
    for scheme, tile in (("two_pass", None), ("fused", None), ("fused", (0, 0, 4))):
        s = Solver(lat, dims, 0.57, faces=faces, wall_u=wall_u, storage=storage, scheme=scheme, force=force,
                   tile=tile)
        s.set_populations(np.ascontiguousarray(f0))
        s.step(12)
        outs.append(s.get_populations())
        s.close()
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[1], outs[2])


@pytest.mark.parametrize("lat,tile,storage", [("D3Q19", (64, 7, 5), "f32"), ("D3Q19", (64, 7, 5), "f16s"),
                                              ("D3Q19", (64, 6, 5), "f32"), ("D3Q27", (32, 10, 4), "f32"),
                                              ("D3Q27", (32, 10, 4), "f16s")])
@pytest.mark.parametrize("fname", ["lid", "periodic", "duct"])
def test_decoupled_export_warps_bitwise(Solver, lat, tile, storage, fname):
    """Brick shapes with dedicated export warps (decoupled from the node
    warps' per-plane barrier through the staged-plane ring) give the same
    bits as the paper's two-pass schedule, on grids spanning many (ragged)
    bricks and ring laps (sweeps of 4-5 planes, 13-23 planes per column)."""
    dims = (150, 30, 23) if lat == "D3Q19" else (70, 33, 13)
    faces, wall_u = faces_for(lat, fname)
    force = (2e-5, 0, 1e-5) if fname == "duct" else (0, 0, 0)
    f0 = random_state(lat, dims, 77)
    outs = []
    for scheme, t in (("two_pass", None), ("fused", tile), ("fused", (tile[0], tile[1], 0))):
        s = Solver(lat, dims, 0.58, faces=faces, wall_u=wall_u, storage=storage, scheme=scheme, force=force, tile=t)
        if scheme == "fused":
            assert s.info()["tile"][:2] == tile[:2]
        s.set_populations(np.ascontiguousarray(f0))
        s.step(9)
        outs.append(s.get_populations())
        s.close()
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], outs[2])


@pytest.mark.parametrize("lat,tile,storage,slots", [("D3Q27", (32, 14, 4), "f32", 2), ("D3Q19", (32, 14, 5), "f32", 3),
                                                    ("D3Q19", (64, 7, 5), "f16s", 4)])
@pytest.mark.parametrize("fname", ["lid", "periodic", "duct"])
def test_barrier_export_warps_bitwise(Solver, lat, tile, storage, slots, fname, monkeypatch):
    """Brick shapes with two dedicated export warps that own no node but pass
    the node warps' per-plane barrier (selected by a negative export-warp
    field of the pipeline request) give the two-pass bits, on grids of many
    ragged bricks and ring laps."""
    from paper_2304_06437_gb300.solver import fused_plan
    dims = (150, 30, 23) if lat == "D3Q19" else (70, 33, 13)
    faces, wall_u = faces_for(lat, fname)
    force = (2e-5, 0, 1e-5) if fname == "duct" else (0, 0, 0)
    f0 = random_state(lat, dims, 79)
    outs = []
    for scheme, t in (("two_pass", None), ("fused", tile), ("fused", (tile[0], tile[1], 0))):
        if scheme == "fused":
            monkeypatch.setenv("LB_FUSED_PIPELINE", "%d,2,-2" % slots)
            assert fused_plan(lat, dims, storage, t)["export_warps"] == -2
        s = Solver(lat, dims, 0.58, faces=faces, wall_u=wall_u, storage=storage, scheme=scheme, force=force, tile=t)
        monkeypatch.delenv("LB_FUSED_PIPELINE", raising=False)
        if scheme == "fused":
            assert s.info()["tile"][:2] == tile[:2] and s.info()["tma_slots"] == slots
        s.set_populations(np.ascontiguousarray(f0))
        s.step(9)
        outs.append(s.get_populations())
        s.close()
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], outs[2])


@pytest.mark.parametrize("lat", ["D3Q19", "D3Q27"])
def test_sweep_length_invariance(Solver, lat):
    """Every brick split along z gives the same bits (a race would not)."""
    dims = (40, 19, 23)
    faces, wall_u = faces_for(lat, "lid_periodic_z")
    f0 = random_state(lat, dims, 17)
    outs = []
    for bz in (0, 3, 8, 11, 23):
        s = Solver(lat, dims, 0.55, faces=faces, wall_u=wall_u, storage="f32", tile=(0, 0, bz))
        s.set_populations(np.ascontiguousarray(f0))
        s.step(9)
        outs.append(s.get_populations())
        s.close()
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)


@pytest.mark.parametrize("lat", LATTICES)
def test_degenerate_sizes(Solver, lat):
    """Single-node-thick and smaller-than-a-brick grids, periodic and walled."""
    cases = [(1, 1, 1), (1, 6, 1), (5, 1, 1)] if dim_of(lat) == 2 else [(1, 1, 1), (1, 9, 1), (3, 1, 7), (2, 2, 2)]
    for dims in cases:
        for fname in ("periodic", "walls"):
            ref, got, cfg, rho, u = _run_pair(Solver, lat, dims, 0.9, fname, "f64", "fused", 3, seed=5)
            assert np.abs(got - ref).max() < 1e-13, (dims, fname)


def test_taylor_green_2d_fp64_and_fp32(Solver):
    """Config: D2Q9 256^2 periodic Taylor-Green, u0 = 0.01, tau = 0.8, 1000 steps."""
    n, tau, steps = 256, 0.8, 1000
    rho, u, pineq = synth.taylor_green_2d(n, u0=0.01, tau=tau)
    cfg = oracle.make_cfg("D2Q9", (n, n, 1), tau)
    ref = oracle.run(cfg, oracle.init(cfg, rho, u, pineq), steps)
    r_ref, u_ref = oracle.moments(cfg, ref)
    for storage in ("f64", "f32"):
        s = Solver("D2Q9", (n, n), tau, storage=storage)
        s.init_moments(rho, np.ascontiguousarray(u), np.ascontiguousarray(pineq))
        s.step(steps)
        r, uu = s.moments()
        s.close()
        assert rel_l2(r, r_ref) < TOL[storage]
        assert rel_l2(uu, u_ref) < TOL[storage], (storage, rel_l2(uu, u_ref))


@pytest.mark.parametrize("lat,case", [("D3Q19", "cavity"), ("D3Q27", "tg")])
def test_64cubed_configs(Solver, lat, case):
    """Parity sizes of the 3D configs: D3Q19 lid-driven cavity (lid 0.05,
    tau 0.52) and D3Q27 periodic Taylor-Green (u0 0.02, tau 0.8), 200 steps."""
    n, steps = 64, 200
    if case == "cavity":
        tau = 0.52
        faces, wall_u = faces_for(lat, "lid")
        rho, u = synth.rest_state((n, n, n), 3)
        pineq = None
    else:
        tau = 0.8
        faces, wall_u = [0] * 6, None
        rho, u, pineq = synth.taylor_green_3d(n, u0=0.02, tau=tau)
    cfg = oracle.make_cfg(lat, (n, n, n), tau, faces=faces, wall_u=wall_u)
    ref = oracle.run(cfg, oracle.init(cfg, rho, u, pineq), steps)
    r_ref, u_ref = oracle.moments(cfg, ref)
    for storage in ("f64", "f32"):
        s = Solver(lat, (n, n, n), tau, faces=faces, wall_u=wall_u, storage=storage)
        s.init_moments(rho, np.ascontiguousarray(u), None if pineq is None else np.ascontiguousarray(pineq))
        s.step(steps)
        r, uu = s.moments()
        s.close()
        assert rel_l2(r, r_ref) < TOL[storage]
        assert rel_l2(uu, u_ref) < TOL[storage], (storage, rel_l2(uu, u_ref))


@pytest.mark.parametrize("lat", LATTICES)
def test_conservation_and_reductions(Solver, lat):
    dims = (48, 40, 1) if dim_of(lat) == 2 else (24, 20, 18)
    d = dim_of(lat)
    rho, u, pineq = synth.smooth_random_state(dims, d, seed=3)
    s = Solver(lat, dims, 0.56, storage="f64")
    s.init_moments(rho, np.ascontiguousarray(u), np.ascontiguousarray(pineq))
    r0 = s.reduce()
    s.step(500)
    r1 = s.reduce(residual=True)
    s.close()
    assert abs(r1["mass"] - r0["mass"]) / r0["mass"] < 1e-13
    assert np.abs(np.array(r1["momentum"]) - np.array(r0["momentum"])).max() < 1e-13 * rho.size
    assert abs(r0["mass"] - rho.sum()) < 1e-9
    assert r1["residual"] == 1.0


def _numpy_reductions(lat, cfg, f, f_prev, force, rho0=1.0):
    """Mass, momentum and the relative velocity residual of oracle states,
    summed with numpy from their definitions (section 2's moments; u =
    (j + F/2)/rho0).  Returns the residual against the exact previous
    velocity and against that velocity rounded to FP32 (the snapshot the
    library keeps)."""
    c = oracle.lattice_tables(lat)[0]
    d = dim_of(lat)
    F = np.asarray(force, float)[:d]

    def vel(g):
        return (c[:, :d].T @ g + 0.5 * F[:, None]) / rho0

    u, up = vel(f), vel(f_prev)
    up32 = up.astype(np.float32).astype(np.float64)
    nu = np.linalg.norm(u)
    return {"mass": f.sum(), "momentum": c[:, :d].T @ f.sum(axis=1),
            "residual": np.linalg.norm(u - up) / nu, "residual_f32prev": np.linalg.norm(u - up32) / nu,
            "unorm": nu, "upnorm": np.linalg.norm(up)}


@pytest.mark.parametrize("lat", LATTICES)
@pytest.mark.parametrize("case", ["periodic_forced_flow", "lid"])
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_reductions_match_numpy_sums(Solver, lat, case, storage):
    """lb_reduce (S6) against numpy sums of the definitions (section 2's
    moments; u = (j + F/2)/rho0): at an oracle state t set from outside, and
    K steps later at the state the GPU reached, read back through
    lb_get_populations -- which the oracle's own state at t + K pins within
    the parity tolerance.  A mean flow (or a driven lid) makes the momentum
    non-zero and changing, so a wrong or constant value fails; the residual is
    compared with ||u_t+K - u_t|| / ||u_t+K||."""
    d = dim_of(lat)
    dims = (40, 28, 1) if d == 2 else (17, 13, 11)
    if case == "lid":
        faces, wall_u = faces_for(lat, "lid")
        force = (0.0, 0.0, 0.0)
    else:
        faces, wall_u = [0] * 6, None
        force = (3e-5, -2e-5, 1e-5)[:d] + (0.0,) * (3 - d)
    cfg = oracle_cfg(lat, dims, 0.62, faces, wall_u, force=force)
    rho, u, pineq = synth.smooth_random_state(dims, d, seed=17)
    u = u + np.array([0.02, -0.013, 0.007][:d])[:, None]
    K = 20
    f_a = oracle.run(cfg, oracle.init(cfg, rho, np.ascontiguousarray(u), pineq), 5)
    f_b_oracle = oracle.run(cfg, f_a, K)
    # the state as stored (FP32 storage rounds each shifted population): the
    # reductions read the stored values, so the numpy sums take the same ones
    w = oracle.lattice_tables(lat)[1]
    f_a = round_populations(f_a, w, storage)
    s = Solver(lat, dims, 0.62, faces=faces, wall_u=wall_u, storage=storage, force=force)
    s.set_populations(np.ascontiguousarray(f_a))
    first = s.reduce(residual=True)
    s.step(K)
    got = s.reduce(residual=True)
    f_b = s.get_populations()
    s.close()
    # the GPU's state at t + K is the oracle's (parity tolerance per population)
    assert np.abs(f_b - f_b_oracle).max() <= {"f64": 1e-13, "f32": 2e-6}[storage]
    want_a = _numpy_reductions(lat, cfg, f_a, f_a, force)
    want = _numpy_reductions(lat, cfg, f_b, f_a, force)
    want_oracle = _numpy_reductions(lat, cfg, f_b_oracle, f_a, force)
    # the first residual has no previous velocity: 1 by definition
    assert first["residual"] == 1.0
    # FP64 sums of the same stored values: rounding order only
    tol = 1e-13
    assert abs(first["mass"] - want_a["mass"]) <= tol * want_a["mass"]
    assert abs(got["mass"] - want["mass"]) <= tol * want["mass"]
    mom_scale = np.abs(want["momentum"]).max()
    assert mom_scale > 1e-3 * f_b.shape[1]  # the momentum is far from zero
    assert np.abs(np.array(got["momentum"]) - want["momentum"]).max() <= tol * mom_scale
    assert np.abs(np.array(first["momentum"]) - want_a["momentum"]).max() <= tol * mom_scale
    assert np.abs(want["momentum"] - want_a["momentum"]).max() > 1e-6 * mom_scale  # it changed over K steps
    # the residual: against the FP32-snapshot definition tightly, and against
    # the exact definition within the snapshot's rounding bound
    # | ||u - fl(up)|| - ||u - up|| | <= ||fl(up) - up|| <= 2^-24 ||up||
    r = got["residual"]
    assert want["residual"] > 1e-4
    rtol = 1e-10
    assert abs(r - want["residual_f32prev"]) <= rtol * want["residual"]
    assert abs(r - want["residual"]) <= 2.0 ** -24 * want["upnorm"] / want["unorm"] + rtol * want["residual"]
    # and against the oracle's own state at t + K, with the same FP32
    # snapshot of u_t (FP64: to rounding; FP32: the per-population error of
    # at most 2e-6 moves u by ~1e-6 relative)
    assert abs(r - want_oracle["residual_f32prev"]) <= {"f64": 1e-9, "f32": 1e-3}[storage] * want_oracle["residual"]


def test_residual_restarts_after_a_state_change(Solver):
    """Setting the state from outside starts a new residual history: the next
    residual call reports 1 (no previous velocity of this history)."""
    dims = (12, 10, 8)
    rho, u, pineq = synth.smooth_random_state(dims, 3, seed=4)
    s = Solver("D3Q19", dims, 0.7, storage="f64")
    s.init_moments(rho, np.ascontiguousarray(u), np.ascontiguousarray(pineq))
    assert s.reduce(residual=True)["residual"] == 1.0
    s.step(3)
    r = s.reduce(residual=True)["residual"]
    assert r > 0.0 and r != 1.0
    s.set_populations(s.get_populations())
    assert s.reduce(residual=True)["residual"] == 1.0
    s.close()


def test_init_moments_device_buffers_and_readback(Solver):
    import torch
    dims = (33, 17, 9)
    rho, u, pineq = synth.smooth_random_state(dims, 3, seed=8)
    s = Solver("D3Q19", dims, 0.7, storage="f64")
    s.init_moments(torch.from_numpy(rho).cuda(), torch.from_numpy(np.ascontiguousarray(u)).cuda(),
                   torch.from_numpy(np.ascontiguousarray(pineq)).cuda())
    rt = torch.empty(rho.size, dtype=torch.float64, device="cuda")
    ut = torch.empty((3, rho.size), dtype=torch.float64, device="cuda")
    s.moments(rt, ut)
    torch.cuda.synchronize()
    assert np.abs(rt.cpu().numpy() - rho).max() < 1e-14
    assert np.abs(ut.cpu().numpy() - u).max() < 1e-15
    cfg = oracle.make_cfg("D3Q19", dims, 0.7)
    fo = oracle.init(cfg, rho, u, pineq)
    assert np.abs(s.get_populations() - fo).max() < 1e-15
    box = s.get_region((3, 4, 5), (6, 2, 3))
    full = s.get_populations().reshape(19, 9, 17, 33)
    assert np.array_equal(box.reshape(19, 3, 2, 6), full[:, 5:8, 4:6, 3:9])
    s.close()


def test_host_moment_fields_cross_in_chunks(Solver):
    """Host moment fields larger than the library's transfer buffer (512 MB:
    3 chunks in with the momentum flux, 2 out) give exactly the bits of the
    same fields passed as device buffers, on both the way in
    (lb_init_moments) and the way out (lb_moments)."""
    import torch
    dims = (272, 256, 256)
    N = dims[0] * dims[1] * dims[2]
    g = torch.Generator(device="cuda").manual_seed(5)
    rho_d = 1.0 + 0.01 * torch.rand(N, dtype=torch.float64, device="cuda", generator=g)
    u_d = 0.02 * (torch.rand((3, N), dtype=torch.float64, device="cuda", generator=g) - 0.5)
    p_d = 1e-4 * (torch.rand((6, N), dtype=torch.float64, device="cuda", generator=g) - 0.5)
    rho_h, u_h, p_h = rho_d.cpu().numpy(), u_d.cpu().numpy(), p_d.cpu().numpy()
    outs = []
    for host in (False, True):
        s = Solver("D3Q19", dims, 0.7, storage="f32")
        if host:
            s.init_moments(rho_h, u_h, p_h)
            r, uu = s.moments()
        else:
            s.init_moments(rho_d, u_d, p_d)
            r = torch.empty(N, dtype=torch.float64, device="cuda")
            uu = torch.empty((3, N), dtype=torch.float64, device="cuda")
            s.moments(r, uu)
            torch.cuda.synchronize()
            r, uu = r.cpu().numpy(), uu.cpu().numpy()
        outs.append((s.get_region((0, 0, 0), dims), r, uu))
        s.close()
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)
    assert np.abs(outs[1][1] - rho_h).max() < 1e-6


@pytest.mark.parametrize("lat,storage", [("D3Q19", "f32"), ("D3Q27", "f16s"), ("D2Q9", "bf16s"), ("D3Q19", "f64")])
def test_checkpoint_resume_is_bitwise(Solver, lat, storage):
    """Checkpoint (lb_get_populations) and resume in a fresh context
    (lb_set_populations, which rebuilds the brick shell) give exactly the
    bits of an uninterrupted run for FP32 / FP16 / BF16 storage: the stored
    shifted values round-trip exactly through f = ft + t_a rho0 in FP64, and
    the shell is a function of the stored state.  FP64 storage loses the
    last bits of ft in that sum, so there the resumed run agrees to rounding."""
    dims = (70, 45, 1) if dim_of(lat) == 2 else (41, 19, 23)
    faces, wall_u = faces_for(lat, "lid")
    f0 = random_state(lat, dims, 61)
    with Solver(lat, dims, 0.66, faces=faces, wall_u=wall_u, storage=storage) as s:
        s.set_populations(np.ascontiguousarray(f0))
        s.step(11)
        want = s.get_populations()
    with Solver(lat, dims, 0.66, faces=faces, wall_u=wall_u, storage=storage) as a:
        a.set_populations(np.ascontiguousarray(f0))
        a.step(4)
        ckpt = a.get_populations()
    with Solver(lat, dims, 0.66, faces=faces, wall_u=wall_u, storage=storage) as b:
        b.set_populations(ckpt)
        b.step(7)
        got = b.get_populations()
    if storage == "f64":
        assert np.abs(got - want).max() < 1e-14
    else:
        assert np.array_equal(got, want)


@pytest.mark.parametrize("storage,pipeline,slots", [("f32", "2,0,-1,0,1", 2)])
@pytest.mark.parametrize("fname", ["lid", "periodic", "duct"])
def test_tma_store_variant_bitwise(Solver, fname, storage, pipeline, slots, monkeypatch):
    """The brick shape whose completed planes leave through a shared-memory
    buffer and one TMA store (64 x 8, two-slot ring; selected by the store
    field of the pipeline request) gives the two-pass bits, including ragged
    bricks whose out-of-range lanes the store drops."""
    lat, dims = "D3Q19", (150, 30, 23)
    faces, wall_u = faces_for(lat, fname)
    force = (2e-5, 0, 1e-5) if fname == "duct" else (0, 0, 0)
    f0 = random_state(lat, dims, 78)
    outs = []
    for scheme, t in (("two_pass", None), ("fused", (64, 8, 5)), ("fused", (64, 8, 0))):
        if scheme == "fused":
            monkeypatch.setenv("LB_FUSED_PIPELINE", pipeline)
        s = Solver(lat, dims, 0.58, faces=faces, wall_u=wall_u, storage=storage, scheme=scheme, force=force, tile=t)
        monkeypatch.delenv("LB_FUSED_PIPELINE", raising=False)
        if scheme == "fused":
            assert s.info()["tma_slots"] == slots and s.info()["tile"][:2] == (64, 8)
        s.set_populations(np.ascontiguousarray(f0))
        s.step(9)
        outs.append(s.get_populations())
        s.close()
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], outs[2])
