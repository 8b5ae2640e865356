"""The two-component colour-gradient step on the GPU (lb_cg_*) against the
FP64 oracle of the same step (oracle.cg_*), through the C ABI.

FP64: populations within 1e-13 after one step, fields within 1e-12 relative
L2 after twenty; FP32: 1e-5.  A static droplet run on the GPU gives the
oracle's pressure jump (Laplace's law is pinned on the oracle).
"""
import numpy as np
import pytest

import oracle
import synth
from lbcase import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import torch
    assert torch.cuda.is_available()
    from paper_2304_06437_gb300 import build
    build.build()
    import paper_2304_06437_gb300 as P
    return P


def _droplet_state(dims, seed):
    d = 2 if dims[2] == 1 else 3
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r = np.sqrt((x - nx / 2.3) ** 2 + (y - ny / 1.9) ** 2 + ((z - nz / 2.1) ** 2 if d == 3 else 0)).ravel()
    phi = np.tanh((min(nx, ny) / 3.0 - r) / 2.0)
    _, u, _ = synth.smooth_random_state(dims, d, seed=seed, du=0.02)
    return (1 + phi) / 2, (1 - phi) / 2, np.ascontiguousarray(u)


CASES = [("D2Q9", (37, 29, 1)), ("D3Q19", (13, 11, 9))]


@pytest.mark.parametrize("lat,dims", CASES)
@pytest.mark.parametrize("storage,ftol,tol", [("f64", 1e-13, 1e-12), ("f32", 2e-6, 1e-5)])
def test_cg_matches_oracle(lb, lat, dims, storage, ftol, tol):
    tau, sigma, beta = 0.8, 0.02, 0.7
    rr, rb, u = _droplet_state(dims, 3)
    cfg = oracle.make_cg_cfg(lat, dims, tau, sigma, beta)
    fr0, fb0 = oracle.cg_init(cfg, rr, rb, u)
    with lb.CGSolver(lat, dims, tau, sigma, beta, storage=storage) as s:
        s.set_populations(np.ascontiguousarray(fr0), np.ascontiguousarray(fb0))
        s.step(1)
        gr, gb = s.get_populations()
        rr1, rb1 = oracle.cg_run(cfg, fr0, fb0, 1)
        assert np.abs(gr - rr1).max() < ftol and np.abs(gb - rb1).max() < ftol
        s.step(19)
        R, Bc, uu = s.fields()
    fr20, fb20 = oracle.cg_run(cfg, fr0, fb0, 20)
    R0, B0, u0 = oracle.cg_fields(cfg, fr20, fb20)
    assert rel_l2(R, R0) < tol and rel_l2(Bc, B0) < tol
    assert rel_l2(uu, u0) < tol, rel_l2(uu, u0)


def test_cg_init_matches_oracle_init(lb):
    lat, dims = "D3Q19", (12, 10, 8)
    rr, rb, u = _droplet_state(dims, 8)
    cfg = oracle.make_cg_cfg(lat, dims, 0.7, 0.01, 0.5)
    fr0, fb0 = oracle.cg_init(cfg, rr, rb, u)
    with lb.CGSolver(lat, dims, 0.7, 0.01, 0.5, storage="f64") as s:
        s.init(rr, rb, u)
        gr, gb = s.get_populations()
        R, Bc, uu = s.fields()
    assert np.abs(gr - fr0).max() < 1e-15 and np.abs(gb - fb0).max() < 1e-15
    assert np.abs(R - rr).max() < 1e-14 and np.abs(uu - u).max() < 1e-14


def test_cg_static_droplet_pressure_jump(lb):
    """2D droplet (R = 12, sigma = 0.01) after 3000 steps: the GPU's pressure
    jump equals the oracle's, which obeys Laplace's law (CPU pin)."""
    n, R, sigma = 64, 12, 0.01
    x, y = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    r = np.sqrt((x - (n - 1) / 2) ** 2 + (y - (n - 1) / 2) ** 2).ravel()
    phi = np.tanh((R - r) / 2.0)
    rr, rb = (1 + phi) / 2, (1 - phi) / 2
    cfg = oracle.make_cg_cfg("D2Q9", (n, n), 1.0, sigma, 0.7)
    fr, fb = oracle.cg_run(cfg, *oracle.cg_init(cfg, rr, rb), 3000)
    Ro, Bo, _ = oracle.cg_fields(cfg, fr, fb)

    def jump(rho):
        rho = rho.reshape(n, n)
        c = n // 2
        return (rho[c - 2:c + 2, c - 2:c + 2].mean() - rho[:4, :4].mean()) / 3.0

    for storage, tol in (("f64", 1e-9), ("f32", 2e-3)):
        with lb.CGSolver("D2Q9", (n, n), 1.0, sigma, 0.7, storage=storage) as s:
            s.init(rr, rb)
            s.step(3000)
            R_, B_, _ = s.fields()
        dp_gpu, dp_ora = jump(R_ + B_), jump(Ro + Bo)
        assert abs(dp_gpu - dp_ora) < tol * abs(dp_ora), (storage, dp_gpu, dp_ora)
        assert abs(dp_gpu * R / sigma - 1) < 0.05


# ------------------------------------------------------------ near-contact
# interactions (section 2.2)

def _droplet_pair(lat, seed):
    """Two unequal droplets facing each other across a thin film (flags
    present), with a small random velocity."""
    if lat == "D2Q9":
        nx, ny = 64, 31
        dims = (nx, ny, 1)
        y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        r1 = np.hypot(x - 21.3, y - 15.2)
        r2 = np.hypot(x - 42.1, y - 16.4)
        R1, R2 = 9.0, 7.0
    else:
        nx, ny, nz = 36, 18, 17
        dims = (nx, ny, nz)
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        r1 = np.sqrt((x - 11.2) ** 2 + (y - 8.7) ** 2 + (z - 8.1) ** 2)
        r2 = np.sqrt((x - 24.6) ** 2 + (y - 9.1) ** 2 + (z - 8.4) ** 2)
        R1, R2 = 5.5, 4.5
    phi = np.maximum(np.tanh((R1 - r1) / 1.5), np.tanh((R2 - r2) / 1.5)).ravel()
    d = 2 if lat == "D2Q9" else 3
    _, u, _ = synth.smooth_random_state(dims, d, seed=seed, du=0.01)
    return dims, (1 + phi) / 2, (1 - phi) / 2, np.ascontiguousarray(u)


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
@pytest.mark.parametrize("storage,ftol,tol", [("f64", 1e-13, 1e-12), ("f32", 2e-6, 1e-5)])
def test_cg_nci_matches_oracle(lb, lat, storage, ftol, tol):
    """With the near-contact force on, the GPU step equals the oracle's
    (flags present in the state, so the forced coefficients are exercised)."""
    # eps = 3/16: the threshold -13/16 is exact in FP32 and FP64, and no
    # phase value of the compared steps comes within 5e-6 of it (about four
    # times the rounding of an FP32 phase value)
    tau, sigma, beta, amp, eps, h = 0.9, 0.01, 0.7, 0.02, 0.1875, 2
    dims, rr, rb, u = _droplet_pair(lat, 12)
    cfg = oracle.make_cg_cfg(lat, dims, tau, sigma, beta, nci_amp=amp, nci_eps=eps, nci_h=h)
    fr0, fb0 = oracle.cg_init(cfg, rr, rb, u)
    R0, B0, _ = oracle.cg_fields(cfg, fr0, fb0)
    assert oracle.cg_nci_flags(cfg, (R0 - B0) / (R0 + B0)).sum() > 0
    # the flags are decisions taken in each side's precision: every phase
    # value of the compared steps lies far enough from the bulk threshold
    # that FP32 and FP64 take the same ones
    fr, fb = fr0, fb0
    for _ in range(20):
        Rk, Bk, _ = oracle.cg_fields(cfg, fr, fb)
        assert np.abs((Rk - Bk) / (Rk + Bk) - (-1.0 + eps)).min() > 5e-6
        fr, fb = oracle.cg_run(cfg, fr, fb, 1)
    with lb.CGSolver(lat, dims, tau, sigma, beta, storage=storage) as s:
        s.set_nci(amp, eps, h)
        s.set_populations(np.ascontiguousarray(fr0), np.ascontiguousarray(fb0))
        s.step(1)
        gr, gb = s.get_populations()
        rr1, rb1 = oracle.cg_run(cfg, fr0, fb0, 1)
        assert np.abs(gr - rr1).max() < ftol and np.abs(gb - rb1).max() < ftol
        s.step(19)
        R, Bc, uu = s.fields()
    R20, B20, u20 = oracle.cg_fields(cfg, *oracle.cg_run(cfg, fr0, fb0, 20))
    assert rel_l2(R, R20) < tol and rel_l2(Bc, B20) < tol
    assert rel_l2(uu, u20) < tol, rel_l2(uu, u20)


def test_cg_nci_off_equals_plain_and_arguments_checked(lb):
    """Amplitude 0 gives the plain step bit for bit; out-of-range parameters
    are rejected."""
    lat = "D2Q9"
    dims, rr, rb, u = _droplet_pair(lat, 13)
    outs = []
    for nci in (None, 0.0):
        with lb.CGSolver(lat, dims, 0.9, 0.01, 0.7, storage="f32") as s:
            if nci is not None:
                s.set_nci(nci, 0.1, 2)
            s.init(rr, rb, u)
            s.step(10)
            outs.append(s.get_populations())
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    with lb.CGSolver(lat, dims, 0.9, 0.01, 0.7, storage="f32") as s:
        for args in ((-1.0, 0.1, 1), (0.01, 0.0, 1), (0.01, 2.0, 1), (0.01, 0.1, 0), (0.01, 0.1, 16)):
            with pytest.raises(RuntimeError):
                s.set_nci(*args)
        s.set_nci(0.01, 0.1, 15)  # 2h = 30 <= 31


def test_cg_nci_keeps_approaching_droplets_apart(lb):
    """FP32 on the GPU: two droplets driven together coalesce without the
    near-contact force and stay apart with it (the oracle shows the same)."""
    nx, ny, R, gap, U = 96, 48, 10.0, 6.0, 0.03
    x, y = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    c1, c2, cy = nx / 2 - gap / 2 - R, nx / 2 + gap / 2 + R, (ny - 1) / 2
    phi = np.maximum(np.tanh((R - np.hypot(x - c1, y - cy)) / 1.5),
                     np.tanh((R - np.hypot(x - c2, y - cy)) / 1.5)).ravel()
    u = np.zeros((2, nx * ny))
    u[0] = np.where(x.ravel() < nx / 2, U, -U) * (phi > -0.5)
    mids = []
    for amp in (0.0, 0.01):
        with lb.CGSolver("D2Q9", (nx, ny), 1.0, 0.01, 0.7, storage="f32") as s:
            s.set_nci(amp, 0.1, 2)
            s.init((1 + phi) / 2, (1 - phi) / 2, u)
            s.step(2000)
            Rr, Bb, _ = s.fields()
        mids.append(((Rr - Bb) / (Rr + Bb)).reshape(ny, nx)[ny // 2, nx // 2 - 1:nx // 2 + 1].max())
    assert mids[0] > 0.9 and mids[1] < -0.5
