"""Plain FP64 CPU oracle for the regularized lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_2304_06437_gb300``) and never imports it.

Two implementations live here:

* ``lbm_oracle.c`` -- the oracle proper: two arrays, collide-then-stream, FP64,
  OpenMP over nodes (paper sections 2-3, Eq. equil, Eq. LBexp, Eq. hermite,
  Eq. pushLB; walls per section 5.1 with the halfway bounce-back reading).
* ``brute.py`` -- an independent numpy brute force for tiny grids that reaches
  the regularized set by a numerical weighted least-squares projection instead
  of the closed form, used to cross-check the C oracle.
* ``lbm_oracle.c`` also holds the two-component colour-gradient step
  (section 2.1: relaxation + perturbation of the total set, recolouring of
  each colour) and its near-contact interactions (section 2.2: flags of the
  nodes around thin films of the continuous phase, a repulsive body force on
  them), written in the paper's order with its readings stated there.
* ``storage.py`` -- round-to-nearest-even of the shifted populations to the
  reduced storage formats (FP16, BF16), from the formats' definitions; with
  ``run_stored`` below it gives the exact reference of a reduced-precision run
  (FP64 arithmetic, rounded storage after every step).

The Python wrapper below only marshals numpy arrays into the C entry points.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblbm_oracle.so")
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_lock = threading.Lock()
_lib = None

D2Q9, D3Q19, D3Q27 = 0, 1, 2
PERIODIC, WALL, MOVING_WALL = 0, 1, 2
LATTICE_NAMES = {"D2Q9": D2Q9, "D3Q19": D3Q19, "D3Q27": D3Q27}


class OrcCfg(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("nz", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("rho0", ctypes.c_double),
        ("force", ctypes.c_double * 3),
        ("face_kind", ctypes.c_int * 6),
        ("wall_u", (ctypes.c_double * 3) * 6),
    ]


class OrcCgCfg(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("nz", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("rho0", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("nci_amp", ctypes.c_double),
        ("nci_eps", ctypes.c_double),
        ("nci_h", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)
            and os.path.getmtime(_SO) >= os.path.getmtime(os.path.join(_HERE, "lbm_oracle.h"))):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.POINTER
            dp = P(ctypes.c_double)
            ip = P(ctypes.c_int)
            L.orc_lattice.argtypes = [ctypes.c_int, ip, dp, ip]
            L.orc_q.argtypes = [ctypes.c_int]
            L.orc_dim.argtypes = [ctypes.c_int]
            L.orc_equilibrium.argtypes = [P(OrcCfg), ctypes.c_double, dp, dp]
            L.orc_collide_node.argtypes = [P(OrcCfg), dp, dp, dp]
            L.orc_project_neq.argtypes = [ctypes.c_int, dp, dp]
            L.orc_init.argtypes = [P(OrcCfg), dp, dp, dp, dp]
            L.orc_run.argtypes = [P(OrcCfg), dp, ctypes.c_long, ctypes.c_int]
            L.orc_moments.argtypes = [P(OrcCfg), dp, dp, dp]
            L.orc_max_threads.argtypes = []
            L.orc_cg_weights.argtypes = [ctypes.c_int, dp]
            L.orc_cg_gradient.argtypes = [P(OrcCgCfg), dp, dp]
            L.orc_cg_init.argtypes = [P(OrcCgCfg), dp, dp, dp, dp, dp]
            L.orc_cg_run.argtypes = [P(OrcCgCfg), dp, dp, ctypes.c_long, ctypes.c_int]
            L.orc_cg_fields.argtypes = [P(OrcCgCfg), dp, dp, dp, dp, dp]
            L.orc_cg_nci_flags.argtypes = [P(OrcCgCfg), dp, ctypes.POINTER(ctypes.c_ubyte)]
            _lib = L
    return _lib


def _dp(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_cfg(lattice, dims, tau, rho0=1.0, force=(0.0, 0.0, 0.0), faces=None, wall_u=None) -> OrcCfg:
    """faces: 6 face kinds (-x,+x,-y,+y,-z,+z); default all periodic."""
    if isinstance(lattice, str):
        lattice = LATTICE_NAMES[lattice]
    c = OrcCfg()
    c.lattice = lattice
    nx, ny, nz = (list(dims) + [1, 1])[:3]
    c.nx, c.ny, c.nz = int(nx), int(ny), int(nz)
    c.tau = float(tau)
    c.rho0 = float(rho0)
    for k in range(3):
        c.force[k] = float(force[k]) if k < len(force) else 0.0
    faces = faces if faces is not None else [PERIODIC] * 6
    for k in range(6):
        c.face_kind[k] = int(faces[k])
        for al in range(3):
            c.wall_u[k][al] = float(wall_u[k][al]) if wall_u is not None else 0.0
    return c


def lattice_tables(lattice):
    if isinstance(lattice, str):
        lattice = LATTICE_NAMES[lattice]
    L = lib()
    q = L.orc_q(lattice)
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q, dtype=np.float64)
    opp = np.zeros(q, dtype=np.int32)
    L.orc_lattice(lattice, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w),
                  opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return c, w, opp


def n_nodes(cfg: OrcCfg) -> int:
    return cfg.nx * cfg.ny * cfg.nz


def equilibrium(cfg: OrcCfg, rho: float, u) -> np.ndarray:
    q = lib().orc_q(cfg.lattice)
    u3 = np.zeros(3)
    u3[: len(u)] = u
    out = np.zeros(q)
    lib().orc_equilibrium(ctypes.byref(cfg), float(rho), _dp(u3), _dp(out))
    return out


def collide_node(cfg: OrcCfg, f: np.ndarray):
    q = lib().orc_q(cfg.lattice)
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(q)
    pineq = np.zeros(6)
    rc = lib().orc_collide_node(ctypes.byref(cfg), _dp(f), _dp(out), _dp(pineq))
    assert rc == 0
    np_ = 3 if lib().orc_dim(cfg.lattice) == 2 else 6
    return out, pineq[:np_]


def project_neq(lattice, g: np.ndarray) -> np.ndarray:
    if isinstance(lattice, str):
        lattice = LATTICE_NAMES[lattice]
    g = np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros_like(g)
    assert lib().orc_project_neq(lattice, _dp(g), _dp(out)) == 0
    return out


def init(cfg: OrcCfg, rho: np.ndarray, u: np.ndarray, pineq: np.ndarray | None = None) -> np.ndarray:
    q = lib().orc_q(cfg.lattice)
    N = n_nodes(cfg)
    rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(N)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1, N)
    if pineq is not None:
        pineq = np.ascontiguousarray(pineq, dtype=np.float64).reshape(-1, N)
    f = np.zeros((q, N))
    rc = lib().orc_init(ctypes.byref(cfg), _dp(rho), _dp(u), _dp(pineq), _dp(f))
    if rc != 0:
        raise ValueError("orc_init rejected the configuration (rc=%d)" % rc)
    return f


def run(cfg: OrcCfg, f: np.ndarray, steps: int, threads: int = 0) -> np.ndarray:
    """Advance a copy of f by `steps`; returns the new array."""
    out = np.ascontiguousarray(f, dtype=np.float64).copy()
    rc = lib().orc_run(ctypes.byref(cfg), _dp(out), int(steps), int(threads))
    if rc != 0:
        raise ValueError("orc_run rejected the configuration (rc=%d)" % rc)
    return out


def moments(cfg: OrcCfg, f: np.ndarray):
    N = n_nodes(cfg)
    d = lib().orc_dim(cfg.lattice)
    f = np.ascontiguousarray(f, dtype=np.float64)
    rho = np.zeros(N)
    u = np.zeros((d, N))
    rc = lib().orc_moments(ctypes.byref(cfg), _dp(f), _dp(rho), _dp(u))
    if rc != 0:
        raise ValueError("orc_moments rejected the configuration (rc=%d)" % rc)
    return rho, u


def run_stored(cfg: OrcCfg, f: np.ndarray, steps: int, storage: str, threads: int = 0) -> np.ndarray:
    """Advance f by `steps`, rounding the stored (shifted) populations to the
    storage format after every step; f itself should already be stored values."""
    from .storage import round_populations
    w = lattice_tables(cfg.lattice)[1]
    out = np.ascontiguousarray(f, dtype=np.float64).copy()
    for _ in range(int(steps)):
        out = round_populations(run(cfg, out, 1, threads), w, storage, cfg.rho0)
    return out


# ------------------------------------------------------------ colour gradient
def make_cg_cfg(lattice, dims, tau, sigma, beta, rho0=1.0, nci_amp=0.0, nci_eps=0.1, nci_h=1) -> OrcCgCfg:
    """Two-component colour-gradient configuration (periodic box); nci_amp > 0
    adds the near-contact interactions of section 2.2 (bulk threshold
    nci_eps, sampling distance nci_h)."""
    if isinstance(lattice, str):
        lattice = LATTICE_NAMES[lattice]
    c = OrcCgCfg()
    c.lattice = lattice
    nx, ny, nz = (list(dims) + [1, 1])[:3]
    c.nx, c.ny, c.nz = int(nx), int(ny), int(nz)
    c.tau, c.rho0, c.sigma, c.beta = float(tau), float(rho0), float(sigma), float(beta)
    c.nci_amp, c.nci_eps, c.nci_h = float(nci_amp), float(nci_eps), int(nci_h)
    return c


def cg_weights(lattice) -> np.ndarray:
    if isinstance(lattice, str):
        lattice = LATTICE_NAMES[lattice]
    B = np.zeros(27)
    q = lib().orc_cg_weights(lattice, _dp(B))
    if q < 0:
        raise ValueError("no colour-gradient weights for this lattice")
    return B[:q]


def cg_gradient(cfg: OrcCgCfg, phi: np.ndarray) -> np.ndarray:
    N = cfg.nx * cfg.ny * cfg.nz
    d = lib().orc_dim(cfg.lattice)
    phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(N)
    g = np.zeros((d, N))
    assert lib().orc_cg_gradient(ctypes.byref(cfg), _dp(phi), _dp(g)) == 0
    return g


def cg_init(cfg: OrcCgCfg, rho_r, rho_b, u=None):
    q = lib().orc_q(cfg.lattice)
    N = cfg.nx * cfg.ny * cfg.nz
    rr = np.ascontiguousarray(rho_r, dtype=np.float64).reshape(N)
    rb = np.ascontiguousarray(rho_b, dtype=np.float64).reshape(N)
    uu = None if u is None else np.ascontiguousarray(u, dtype=np.float64).reshape(-1, N)
    fr, fb = np.zeros((q, N)), np.zeros((q, N))
    if lib().orc_cg_init(ctypes.byref(cfg), _dp(rr), _dp(rb), _dp(uu), _dp(fr), _dp(fb)) != 0:
        raise ValueError("orc_cg_init rejected the configuration")
    return fr, fb


def cg_run(cfg: OrcCgCfg, fr, fb, steps: int, threads: int = 0):
    """Advance copies of (f_R, f_B) by `steps`; returns the new pair."""
    fr = np.ascontiguousarray(fr, dtype=np.float64).copy()
    fb = np.ascontiguousarray(fb, dtype=np.float64).copy()
    if lib().orc_cg_run(ctypes.byref(cfg), _dp(fr), _dp(fb), int(steps), int(threads)) != 0:
        raise ValueError("orc_cg_run rejected the configuration")
    return fr, fb


def cg_fields(cfg: OrcCgCfg, fr, fb):
    """(rho_R, rho_B, u) of a two-component state; u = sum (f_R + f_B) c / rho0."""
    N = cfg.nx * cfg.ny * cfg.nz
    d = lib().orc_dim(cfg.lattice)
    rr, rb, u = np.zeros(N), np.zeros(N), np.zeros((d, N))
    assert lib().orc_cg_fields(ctypes.byref(cfg), _dp(np.ascontiguousarray(fr)), _dp(np.ascontiguousarray(fb)),
                               _dp(rr), _dp(rb), _dp(u)) == 0
    return rr, rb, u


def cg_nci_flags(cfg: OrcCgCfg, phi) -> np.ndarray:
    """Near-contact flags (uint8, 1 = force acts) of a phase field (section 2.2)."""
    N = cfg.nx * cfg.ny * cfg.nz
    phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(N)
    fl = np.zeros(N, dtype=np.uint8)
    if lib().orc_cg_nci_flags(ctypes.byref(cfg), _dp(phi), fl.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))) != 0:
        raise ValueError("orc_cg_nci_flags rejected the configuration")
    return fl


def max_threads() -> int:
    return int(lib().orc_max_threads())
