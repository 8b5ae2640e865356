"""Seeded synthetic inputs for the lattice Boltzmann workloads.

This module only produces macroscopic fields (density, velocity, the initial
non-equilibrium stress of an analytic flow) and raw random numbers.  It holds
none of the lattice Boltzmann arithmetic: both the CUDA library and the CPU
oracle turn these fields into populations with their own code.

Layouts follow the library: node index idx = x + nx*(y + ny*z); vectors are
[d][N]; symmetric tensors [3][N] in 2D (xx, yy, xy) and [6][N] in 3D
(xx, yy, zz, xy, xz, yz).  Lattice units throughout (dx = dt = 1, cs^2 = 1/3).

Workloads (the paper has no dataset; every input is analytic or seeded):
  * Taylor-Green vortex, 2D and 3D, periodic box;
  * lid-driven cavity started from rest;
  * body-force-driven channel started from the analytic parabola;
  * smooth random states and raw uniform noise for algebra tests.
"""
from __future__ import annotations

import math

import numpy as np

SEED = 20230412
CS2 = 1.0 / 3.0


def rng(seed: int = SEED) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _grid(dims):
    nx, ny, nz = (list(dims) + [1, 1])[:3]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.reshape(-1).astype(float), y.reshape(-1).astype(float), z.reshape(-1).astype(float)


def taylor_green_2d(n: int, u0: float = 0.01, rho0: float = 1.0, tau: float = 0.8, ny: int | None = None):
    """2D Taylor-Green vortex on an n x ny periodic box (k = 2 pi / n).

    u = -u0 cos(kx) sin(ky), v = u0 sin(kx) cos(ky),
    p = -rho0 u0^2 / 4 (cos 2kx + cos 2ky), rho = rho0 + p / cs2,
    Pi^neq = -rho0 cs2 tau (grad u + grad u^T)  (Navier-Stokes-level stress).
    The velocity amplitude decays as exp(-2 nu k^2 t) with nu = cs2 (tau - 1/2).
    """
    ny = n if ny is None else ny
    x, y, _ = _grid((n, ny, 1))
    k = 2.0 * math.pi / n
    ky = 2.0 * math.pi / ny
    u = -u0 * np.cos(k * x) * np.sin(ky * y)
    v = u0 * np.sin(k * x) * np.cos(ky * y)
    p = -rho0 * u0 * u0 / 4.0 * (np.cos(2 * k * x) + np.cos(2 * ky * y))
    rho = rho0 + p / CS2
    dudx = u0 * k * np.sin(k * x) * np.sin(ky * y)
    dudy = -u0 * ky * np.cos(k * x) * np.cos(ky * y)
    dvdx = u0 * k * np.cos(k * x) * np.cos(ky * y)
    dvdy = -u0 * ky * np.sin(k * x) * np.sin(ky * y)
    s = -rho0 * CS2 * tau
    pineq = np.stack([s * 2 * dudx, s * 2 * dvdy, s * (dudy + dvdx)])
    return rho, np.stack([u, v]), pineq


def taylor_green_2d_mode(n: int, ny: int | None = None):
    """Unit-amplitude velocity mode of taylor_green_2d, for projecting u(t)."""
    ny = n if ny is None else ny
    x, y, _ = _grid((n, ny, 1))
    k = 2.0 * math.pi / n
    ky = 2.0 * math.pi / ny
    return np.stack([-np.cos(k * x) * np.sin(ky * y), np.sin(k * x) * np.cos(ky * y)])


def taylor_green_3d(n: int, u0: float = 0.02, rho0: float = 1.0, tau: float = 0.8):
    """3D Taylor-Green vortex on an n^3 periodic box (k = 2 pi / n).

    u = u0 sin kx cos ky cos kz, v = -u0 cos kx sin ky cos kz, w = 0,
    p = rho0 u0^2 / 16 (cos 2kx + cos 2ky)(cos 2kz + 2), rho = rho0 + p / cs2,
    Pi^neq = -rho0 cs2 tau (grad u + grad u^T).
    """
    x, y, z = _grid((n, n, n))
    k = 2.0 * math.pi / n
    sx, cx = np.sin(k * x), np.cos(k * x)
    sy, cy = np.sin(k * y), np.cos(k * y)
    sz, cz = np.sin(k * z), np.cos(k * z)
    u = u0 * sx * cy * cz
    v = -u0 * cx * sy * cz
    w = np.zeros_like(u)
    p = rho0 * u0 * u0 / 16.0 * (np.cos(2 * k * x) + np.cos(2 * k * y)) * (np.cos(2 * k * z) + 2.0)
    rho = rho0 + p / CS2
    # velocity gradient components d_i u_j
    dudx, dudy, dudz = u0 * k * cx * cy * cz, -u0 * k * sx * sy * cz, -u0 * k * sx * cy * sz
    dvdx, dvdy, dvdz = u0 * k * sx * sy * cz, -u0 * k * cx * cy * cz, u0 * k * cx * sy * sz
    s = -rho0 * CS2 * tau
    pineq = np.stack([
        s * 2 * dudx, s * 2 * dvdy, np.zeros_like(u),
        s * (dudy + dvdx), s * dudz, s * dvdz,
    ])
    return rho, np.stack([u, v, w]), pineq


def rest_state(dims, d: int, rho0: float = 1.0):
    """Fluid at rest (the lid-driven cavity's initial condition)."""
    nx, ny, nz = (list(dims) + [1, 1])[:3]
    N = nx * ny * nz
    return np.full(N, rho0), np.zeros((d, N))


def poiseuille_profile(H: int, F: float, rho0: float, nu: float):
    """Analytic channel profile with walls half a link outside nodes 0 and H-1:
    u_x(y) = F / (2 rho0 nu) (y + 1/2)(H - 1/2 - y), y = 0..H-1."""
    y = np.arange(H, dtype=float)
    return F / (2.0 * rho0 * nu) * (y + 0.5) * (H - 0.5 - y)


def channel_state(dims, F: float, rho0: float, nu: float, d: int):
    """Channel along x with walls on +-y, started from the analytic parabola."""
    nx, ny, nz = (list(dims) + [1, 1])[:3]
    x, y, z = _grid((nx, ny, nz))
    prof = poiseuille_profile(ny, F, rho0, nu)
    N = nx * ny * nz
    u = np.zeros((d, N))
    u[0] = prof[y.astype(int)]
    return np.full(N, rho0), u


def smooth_random_state(dims, d: int, seed: int = SEED, du: float = 0.02, drho: float = 0.01,
                        dpi: float = 1e-3, modes: int = 3):
    """Smooth random fields: a few random Fourier modes per component."""
    g = rng(seed)
    nx, ny, nz = (list(dims) + [1, 1])[:3]
    x, y, z = _grid((nx, ny, nz))

    def field(amp):
        out = np.zeros_like(x)
        for _ in range(modes):
            kx, ky, kz = g.integers(0, 3, size=3)
            ph = g.uniform(0, 2 * math.pi)
            out += amp * g.uniform(-1, 1) * np.cos(2 * math.pi * (kx * x / nx + ky * y / ny + kz * z / nz) + ph)
        return out / modes

    rho = 1.0 + field(drho)
    u = np.stack([field(du) for _ in range(d)])
    npi = 3 if d == 2 else 6
    pineq = np.stack([field(dpi) for _ in range(npi)])
    return rho, u, pineq


def uniform_noise(shape, seed: int = SEED) -> np.ndarray:
    """Raw U(-1, 1) numbers (e.g. to perturb populations beyond the Hermite span)."""
    return rng(seed).uniform(-1.0, 1.0, size=shape)


# ------------------------------------------------------------------ on device
# The same analytic fields generated with torch on the GPU, for grids too large
# to build on the host (e.g. 512^3).  Same formulas as the numpy versions.
def taylor_green_3d_torch(n: int, u0: float, rho0: float, tau: float, torch, device="cuda", pineq=True):
    """taylor_green_3d on the device.  Every field is an outer product of 1D
    sine / cosine vectors, so each output is allocated once (1024^3 fits)."""
    k = 2.0 * math.pi / n
    ar = torch.arange(n, device=device, dtype=torch.float64) * k
    s1, c1 = torch.sin(ar), torch.cos(ar)
    sx, cx = s1.view(1, 1, n), c1.view(1, 1, n)
    sy, cy = s1.view(1, n, 1), c1.view(1, n, 1)
    sz, cz = s1.view(n, 1, 1), c1.view(n, 1, 1)
    N = n * n * n
    u = torch.empty((3, N), device=device, dtype=torch.float64)
    u[0].view(n, n, n).copy_((u0 * sx * cy) * cz)
    u[1].view(n, n, n).copy_((-u0 * cx * sy) * cz)
    u[2].zero_()
    c2 = torch.cos(2.0 * ar)
    rho = ((c2.view(1, 1, n) + c2.view(1, n, 1)) * (rho0 * u0 * u0 / 16.0 / CS2)) * (c2.view(n, 1, 1) + 2.0)
    rho = (rho + rho0).reshape(N)
    if not pineq:
        return rho.contiguous(), u, None
    s = -rho0 * CS2 * tau
    pi = torch.zeros((6, N), device=device, dtype=torch.float64)
    # d_x u = u0 k cx cy cz, d_y v = -u0 k cx cy cz; d_y u + d_x v = 0
    pi[0].view(n, n, n).copy_((s * 2 * u0 * k * cx * cy) * cz)
    pi[1].copy_(-pi[0])
    pi[4].view(n, n, n).copy_((s * (-u0 * k) * sx * cy) * sz)  # d_z u
    pi[5].view(n, n, n).copy_((s * u0 * k * cx * sy) * sz)  # d_z v
    return rho.contiguous(), u, pi


def taylor_green_2d_torch(n: int, u0: float, rho0: float, tau: float, torch, device="cuda"):
    k = 2.0 * math.pi / n
    ar = torch.arange(n, device=device, dtype=torch.float64)
    y, x = torch.meshgrid(ar, ar, indexing="ij")
    u = torch.stack([-u0 * torch.cos(k * x) * torch.sin(k * y), u0 * torch.sin(k * x) * torch.cos(k * y)]).reshape(2, -1)
    p = -rho0 * u0 * u0 / 4.0 * (torch.cos(2 * k * x) + torch.cos(2 * k * y))
    rho = (rho0 + p / CS2).reshape(-1)
    s = -rho0 * CS2 * tau
    dudx = u0 * k * torch.sin(k * x) * torch.sin(k * y)
    pineq = torch.stack([s * 2 * dudx, -s * 2 * dudx, torch.zeros_like(x)]).reshape(3, -1)
    return rho.contiguous(), u.contiguous(), pineq.contiguous()
