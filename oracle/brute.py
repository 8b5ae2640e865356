"""Independent numpy brute force of one regularized lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Written separately
from ``lbm_oracle.c`` to cross-check it on tiny grids: it builds its own
lattice tables and reaches every Hermite-space object numerically instead of
through the closed forms the C oracle uses:

* the order-2 Hermite span (paper Eq. hermite) is the column space of
  ``w_a * H(c_a)`` with H = [1, c_alpha, c_alpha c_beta - cs2 delta];
* an element of that span is fixed by its Hermite moments; we solve the
  normal equations of the weighted least-squares problem for it;
* the regularized non-equilibrium set (paper section 3) is the weighted
  least-squares projection of f - f^eq onto the span;
* the He-Luo equilibrium (Eq. equil) is the span element whose Hermite moments
  are (rho, rho0 u, rho0 u u);
* the forcing reading adds the span element with moments
  (0, (1 - omega/2) F, (1 - omega/2)(u F + F u)).

Streaming is a node-by-node Python loop (pull form of Eq. pushLB, periodic
wrap, halfway bounce-back with the tie-break stated in lbm_oracle.c).  Use only
for grids of a few thousand nodes.
"""
from __future__ import annotations

import itertools

import numpy as np

CS2 = 1.0 / 3.0
_WEIGHTS = {
    "D2Q9": {0: 4 / 9, 1: 1 / 9, 2: 1 / 36},
    "D3Q19": {0: 1 / 3, 1: 1 / 18, 2: 1 / 36},
    "D3Q27": {0: 8 / 27, 1: 2 / 27, 2: 1 / 54, 3: 1 / 216},
}


def lattice(name: str):
    d = 2 if name == "D2Q9" else 3
    vels = []
    for v in itertools.product((-1, 0, 1), repeat=d):
        v = tuple(v) + (0,) * (3 - d)
        if sum(x * x for x in v) in _WEIGHTS[name]:
            vels.append(v)
    vels.sort(key=lambda v: (sum(x * x for x in v), v))
    c = np.array(vels, dtype=np.int64)
    w = np.array([_WEIGHTS[name][int((v * v).sum())] for v in c])
    opp = np.array([next(j for j, v2 in enumerate(c) if (v2 == -v).all()) for v in c])
    return c, w, opp, d


def hermite_matrix(c: np.ndarray, d: int) -> np.ndarray:
    """Columns: H0 = 1, H1 = c_alpha, H2 = c_alpha c_beta - cs2 delta (alpha <= beta)."""
    cols = [np.ones(len(c))]
    for al in range(d):
        cols.append(c[:, al].astype(float))
    for al in range(d):
        for be in range(al, d):
            cols.append(c[:, al] * c[:, be] - (CS2 if al == be else 0.0))
    return np.stack(cols, axis=1)


def _moment_vector(d, m0, m1, m2):
    """Pack (scalar, vector, symmetric tensor) in the column order of hermite_matrix."""
    out = [m0] + [m1[al] for al in range(d)]
    for al in range(d):
        for be in range(al, d):
            out.append(m2[al][be])
    return np.array(out, dtype=float)


class BruteLB:
    def __init__(self, name, dims, tau, rho0=1.0, force=(0, 0, 0), faces=(0,) * 6, wall_u=None):
        self.name = name
        self.c, self.w, self.opp, self.d = lattice(name)
        self.q = len(self.c)
        self.dims = tuple(int(v) for v in (list(dims) + [1, 1])[:3])
        self.tau = float(tau)
        self.omega = 1.0 / self.tau
        self.rho0 = float(rho0)
        self.F = np.array(list(force) + [0.0] * (3 - len(force)), dtype=float)[:3]
        self.faces = list(faces)
        self.wall_u = np.zeros((6, 3)) if wall_u is None else np.array(wall_u, dtype=float)
        self.H = hermite_matrix(self.c, self.d)
        self.B = self.w[:, None] * self.H           # span generators
        self.G = self.H.T @ self.B                   # Gram matrix  H^T W H

    # element of the span with prescribed Hermite moments H^T g = m
    def span_element(self, m):
        return self.B @ np.linalg.solve(self.G, m)

    # weighted least-squares projection onto the span, <x, y> = sum x y / w
    def project(self, g):
        return self.B @ np.linalg.solve(self.G, self.H.T @ g)

    def node_collide(self, f):
        d = self.d
        rho = f.sum()
        j = (f[:, None] * self.c[:, :3]).sum(axis=0).astype(float)
        u = (j + 0.5 * self.F) / self.rho0
        uu = np.outer(u, u)
        feq = self.span_element(_moment_vector(d, rho, self.rho0 * u, self.rho0 * uu))
        fhat = self.project(f - feq)
        g = 1.0 - 0.5 * self.omega
        uF = np.outer(u, self.F) + np.outer(self.F, u)
        S = self.span_element(_moment_vector(d, 0.0, g * self.F, g * uF))
        return feq + (1.0 - self.omega) * fhat + S

    def step(self, f):
        nx, ny, nz = self.dims
        N = nx * ny * nz
        f = np.asarray(f, dtype=float).reshape(self.q, N)
        fpc = np.empty_like(f)
        for i in range(N):
            fpc[:, i] = self.node_collide(f[:, i])
        out = np.empty_like(f)
        n = (nx, ny, nz)
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    i = x + nx * (y + ny * z)
                    p = (x, y, z)
                    for a in range(self.q):
                        s = [p[k] - int(self.c[a, k]) for k in range(3)]
                        crossed = []
                        for k in range(3):
                            if s[k] < 0 or s[k] >= n[k]:
                                face = 2 * k + (0 if s[k] < 0 else 1)
                                if self.faces[face] == 0:
                                    s[k] %= n[k]
                                else:
                                    crossed.append(face)
                        if crossed:
                            if any(self.faces[fc] == 1 for fc in crossed):
                                uw = np.zeros(3)
                            else:
                                uw = self.wall_u[min(crossed)]
                            out[a, i] = fpc[self.opp[a], i] + 2.0 * self.w[a] * self.rho0 * float(self.c[a] @ uw) / CS2
                        else:
                            out[a, i] = fpc[a, s[0] + nx * (s[1] + ny * s[2])]
        return out

    def run(self, f, steps):
        for _ in range(steps):
            f = self.step(f)
        return f

    def moments(self, f):
        f = np.asarray(f, dtype=float)
        rho = f.sum(axis=0)
        j = np.einsum("aN,ak->kN", f, self.c[:, :3].astype(float))
        u = (j + 0.5 * self.F[:, None]) / self.rho0
        return rho, u[: self.d]
