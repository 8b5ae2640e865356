"""Shared test helpers: one description of a case drives both the CUDA
library (through the C ABI) and the CPU oracle, with identical seeded inputs."""
from __future__ import annotations

import numpy as np

import oracle
import synth

FACE_SETS = {
    "periodic": ([0] * 6, None),
    "walls": ([1] * 6, None),
    "lid": ([1, 1, 1, 2, 1, 1], [[0, 0, 0]] * 3 + [[0.05, 0, 0]] + [[0, 0, 0]] * 2),
    "duct": ([0, 0, 1, 1, 1, 1], None),
    "lid_periodic_z": ([1, 1, 1, 2, 0, 0], [[0, 0, 0]] * 3 + [[0.04, 0, 0.01]] + [[0, 0, 0]] * 2),
}


def dim_of(lat):
    return 2 if lat == "D2Q9" else 3


def faces_for(lat, name):
    faces, wall_u = FACE_SETS[name]
    faces = list(faces)
    if dim_of(lat) == 2:
        faces = faces[:4] + [0, 0]
    return faces, wall_u


def rel_l2(a, b):
    a = np.asarray(a, float).ravel()
    b = np.asarray(b, float).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def random_state(lat, dims, seed, noise=2e-3):
    """Smooth random moments plus population noise beyond the Hermite span,
    built on the oracle side; the same populations are handed to the GPU."""
    d = dim_of(lat)
    cfg = oracle.make_cfg(lat, dims, 0.7)
    rho, u, pineq = synth.smooth_random_state(dims, d, seed=seed)
    f = oracle.init(cfg, rho, u, pineq)
    w = oracle.lattice_tables(lat)[1]
    return f + noise * w[:, None] * synth.uniform_noise(f.shape, seed=seed + 1)


def oracle_cfg(lat, dims, tau, faces, wall_u, force=(0, 0, 0), rho0=1.0):
    return oracle.make_cfg(lat, dims, tau, rho0=rho0, force=force, faces=faces, wall_u=wall_u)
