"""Thin Python front end of the C ABI (include/lb.h).

Only marshals arguments: every step of the method runs in the CUDA library.
numpy arrays are passed as host buffers; torch CUDA tensors as device
buffers (PyTorch provides device memory and streams, nothing else).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _binding as B


def _is_torch_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def _ptr(x, dtype=np.float64):
    """(pointer, on_device) of a contiguous FP64 buffer.

    A torch CUDA tensor is handed over as a device pointer after the torch
    stream that produced it has finished: the library reads and writes it on
    its own stream, which is not ordered after torch's (without this wait the
    library could read a tensor whose producing kernels are still running, or
    overwrite memory that queued torch work still uses)."""
    if x is None:
        return None, 0
    if _is_torch_cuda(x):
        import torch
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise ValueError("device buffers must be contiguous torch.float64 tensors")
        torch.cuda.current_stream(x.device).synchronize()
        return ctypes.c_void_p(x.data_ptr()), 1
    if not (isinstance(x, np.ndarray) and x.dtype == dtype and x.flags["C_CONTIGUOUS"]):
        raise ValueError("host buffers must be C-contiguous float64 numpy arrays")
    return ctypes.c_void_p(x.ctypes.data), 0


class Solver:
    """One lattice Boltzmann domain resident on the GPU.

    lattice: "D2Q9" | "D3Q19" | "D3Q27"; dims: (nx, ny[, nz]); tau > 1/2;
    faces: six face kinds (-x,+x,-y,+y,-z,+z) from {"periodic","wall",
    "moving_wall"} or ints; wall_u: 6x3 wall velocities; storage: "f64" |
    "f32" | "f16s" | "bf16s"; scheme: "fused" | "two_pass".
    """

    _FACE = {"periodic": B.LB_PERIODIC, "wall": B.LB_WALL, "moving_wall": B.LB_MOVING_WALL}

    def __init__(self, lattice, dims, tau, faces=None, wall_u=None, storage="f32", scheme="fused",
                 rho0=1.0, force=(0.0, 0.0, 0.0), stream=None, tile=None, device=-1):
        self._lib = B.load()
        self._ctx = ctypes.c_void_p()
        self._owned = True
        self.lattice = lattice
        self.lat_id = B.LATTICES[lattice] if isinstance(lattice, str) else int(lattice)
        d = 2 if self.lat_id == B.LB_D2Q9 else 3
        dims = list(dims) + [1] * (3 - len(dims))
        self.dims = tuple(int(v) for v in dims[:3])
        self.d = d
        self.q = {0: 9, 1: 19, 2: 27}[self.lat_id]
        self.n = self.dims[0] * self.dims[1] * self.dims[2]
        bnd = B.lb_boundary()
        faces = faces if faces is not None else [B.LB_PERIODIC] * 6
        for k in range(6):
            fk = faces[k] if k < len(faces) else B.LB_PERIODIC
            bnd.kind[k] = self._FACE[fk] if isinstance(fk, str) else int(fk)
            for al in range(3):
                bnd.wall_u[k][al] = float(wall_u[k][al]) if wall_u is not None else 0.0
        opt = B.lb_options()
        self._lib.lb_default_options(ctypes.byref(opt))
        opt.storage = B.STORAGES[storage] if isinstance(storage, str) else int(storage)
        opt.scheme = B.SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
        opt.rho0 = float(rho0)
        for k in range(3):
            opt.force[k] = float(force[k]) if k < len(force) else 0.0
        if stream is not None:
            opt.stream = ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        if tile is not None:
            for k in range(3):
                opt.tile[k] = int(tile[k]) if k < len(tile) else 0
        opt.device = int(device)
        self.rho0 = float(rho0)
        dims_arr = (ctypes.c_int64 * 3)(*self.dims)
        B.check(self._lib.lb_create(self.lat_id, dims_arr, float(tau), ctypes.byref(bnd), ctypes.byref(opt),
                                    ctypes.byref(self._ctx)), "lb_create")

    # ------------------------------------------------------------ lifetime
    @classmethod
    def _view(cls, ctx_ptr, lattice, dims, rho0=1.0):
        """A non-owning Solver over a context that something else (a slab
        group) owns and destroys."""
        self = cls.__new__(cls)
        self._lib = B.load()
        self._ctx = ctypes.c_void_p(ctx_ptr)
        self._owned = False
        self.lattice = lattice
        self.lat_id = B.LATTICES[lattice] if isinstance(lattice, str) else int(lattice)
        self.d = 2 if self.lat_id == B.LB_D2Q9 else 3
        self.q = {0: 9, 1: 19, 2: 27}[self.lat_id]
        self.dims = tuple(int(v) for v in (list(dims) + [1] * 3)[:3])
        self.n = self.dims[0] * self.dims[1] * self.dims[2]
        self.rho0 = float(rho0)
        return self

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            if getattr(self, "_owned", True):
                self._lib.lb_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------ state
    def init_moments(self, rho, u, pineq=None):
        pr, dev = _ptr(rho)
        pu, dev2 = _ptr(u)
        pp, dev3 = _ptr(pineq)
        if pineq is None:
            dev3 = dev
        if not (dev == dev2 == dev3):
            raise ValueError("rho, u and pineq must all be host or all be device buffers")
        B.check(self._lib.lb_init_moments(self._ctx, pr, pu, pp, dev), "lb_init_moments")

    def init_uniform(self, rho, u=(0.0, 0.0, 0.0)):
        uu = (ctypes.c_double * 3)(*(list(u) + [0.0] * 3)[:3])
        B.check(self._lib.lb_init_uniform(self._ctx, float(rho), uu), "lb_init_uniform")

    def set_populations(self, f):
        p, dev = _ptr(f)
        B.check(self._lib.lb_set_populations(self._ctx, p, dev), "lb_set_populations")

    def get_populations(self, out=None):
        out = np.empty((self.q, self.n)) if out is None else out
        p, dev = _ptr(out)
        B.check(self._lib.lb_get_populations(self._ctx, p, dev), "lb_get_populations")
        return out

    def get_region(self, lo, size):
        lo3 = (list(lo) + [0, 0, 0])[:3]
        sz3 = (list(size) + [1, 1, 1])[:3]
        out = np.empty((self.q, sz3[0] * sz3[1] * sz3[2]))
        B.check(self._lib.lb_get_region(self._ctx, (ctypes.c_int64 * 3)(*lo3), (ctypes.c_int64 * 3)(*sz3),
                                        ctypes.c_void_p(out.ctypes.data)), "lb_get_region")
        return out

    # ------------------------------------------------------------ stepping
    def step(self, n=1):
        B.check(self._lib.lb_step(self._ctx, int(n)), "lb_step")

    def sync(self):
        B.check(self._lib.lb_sync(self._ctx), "lb_sync")

    def moments(self, rho=None, u=None):
        """Returns (rho [N], u [d][N]); pass torch CUDA tensors to stay on device."""
        if rho is None and u is None:
            rho = np.empty(self.n)
            u = np.empty((self.d, self.n))
        pr, dev = _ptr(rho)
        pu, dev2 = _ptr(u)
        if rho is not None and u is not None and dev != dev2:
            raise ValueError("rho and u must both be host or both be device buffers")
        B.check(self._lib.lb_moments(self._ctx, pr, pu, dev if rho is not None else dev2), "lb_moments")
        return rho, u

    def reduce(self, residual=False):
        mass = ctypes.c_double()
        mom = (ctypes.c_double * 3)()
        res = ctypes.c_double()
        rc = self._lib.lb_reduce(self._ctx, ctypes.byref(mass), mom, ctypes.byref(res) if residual else None)
        B.check(rc, "lb_reduce")
        out = {"mass": mass.value, "momentum": [mom[0], mom[1], mom[2]][: self.d]}
        if residual:
            out["residual"] = res.value
        return out

    def autotune(self, steps=5):
        """Time every compiled brick shape on a proxy of this domain and switch
        to the fastest (lb_autotune); returns the timing table (empty when the
        choice came from the cache)."""
        cap = 64
        tab = (B.lb_tune_entry * cap)()
        n = ctypes.c_int32()
        B.check(self._lib.lb_autotune(self._ctx, int(steps), tab, cap, ctypes.byref(n)), "lb_autotune")
        return [{name: getattr(tab[i], name) for name, _ in tab[i]._fields_} for i in range(n.value)]

    # ------------------------------------------------------------ slab halos
    def halo_bytes(self) -> int:
        n = ctypes.c_int64()
        B.check(self._lib.lb_halo_bytes(self._ctx, ctypes.byref(n)), "lb_halo_bytes")
        return n.value

    def halo_pack(self, side, buf):
        """Enqueue the records leaving through link face `side` (0 low, 1
        high) into buf, a contiguous CUDA tensor of halo_bytes() bytes."""
        B.check(self._lib.lb_halo_pack(self._ctx, int(side), ctypes.c_void_p(buf.data_ptr())), "lb_halo_pack")

    def halo_unpack(self, side, buf):
        """Enqueue the copy of a neighbour's message into the ghost records of
        link face `side`."""
        B.check(self._lib.lb_halo_unpack(self._ctx, int(side), ctypes.c_void_p(buf.data_ptr())), "lb_halo_unpack")

    def info(self) -> dict:
        inf = B.lb_info_t()
        B.check(self._lib.lb_info(self._ctx, ctypes.byref(inf)), "lb_info")
        return {
            "lattice": inf.lattice, "q": inf.q, "d": inf.d, "storage": inf.storage, "scheme": inf.scheme,
            "dims": tuple(inf.dims), "steps_done": inf.steps_done, "tile": tuple(inf.tile),
            "population_bytes": inf.population_bytes, "aux_bytes": inf.aux_bytes,
            "algorithmic_bytes_per_update": inf.algorithmic_bytes_per_update,
            "nodes_per_thread": inf.nodes_per_thread, "tma_slots": inf.tma_slots,
        }


class Batch:
    """Many Solver domains stepped together (lb_batch_*): one persistent
    launch per brick-shape class and time step, two steps per CUDA graph
    replay.  The solvers must stay open while the batch exists."""

    def __init__(self, solvers, stream=None):
        self._lib = B.load()
        self.solvers = list(solvers)
        arr = (ctypes.c_void_p * len(self.solvers))(*[s._ctx.value for s in self.solvers])
        st = ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream))) if stream is not None else None
        self._b = ctypes.c_void_p()
        B.check(self._lib.lb_batch_create(arr, len(self.solvers), st, ctypes.byref(self._b)), "lb_batch_create")

    def step(self, n=1):
        B.check(self._lib.lb_batch_step(self._b, int(n)), "lb_batch_step")

    def sync(self):
        B.check(self._lib.lb_batch_sync(self._b), "lb_batch_sync")

    def reduce(self, residual=False):
        """lb_reduce of every member in one pass (lb_batch_reduce): a list of
        dicts in member order, with "diverged" set where a value is not
        finite."""
        n = len(self.solvers)
        out = np.zeros(6 * n)
        B.check(self._lib.lb_batch_reduce(self._b, 1 if residual else 0,
                                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "lb_batch_reduce")
        res = []
        for i, s in enumerate(self.solvers):
            o = out[6 * i:6 * i + 6]
            r = {"mass": float(o[0]), "momentum": [float(v) for v in o[1:4]][: s.d], "diverged": o[5] != 0}
            if residual:
                r["residual"] = float(o[4])
            res.append(r)
        return res

    def info(self) -> dict:
        inf = B.lb_batch_info_t()
        B.check(self._lib.lb_batch_info(self._b, ctypes.byref(inf)), "lb_batch_info")
        return {name: getattr(inf, name) for name, _ in inf._fields_}

    def close(self):
        if getattr(self, "_b", None) and self._b.value:
            self._lib.lb_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class SlabGroup:
    """One domain cut into slabs along its slowest axis (z in 3D, y in 2D),
    one context and stream per rank, halos exchanged on the device between
    steps (lb_group_*): the decomposition of a multi-GPU run, in one process.
    Initialisation and readout split or join the canonical arrays by the
    ranks' node ranges (a slab is a contiguous range of nodes)."""

    def __init__(self, lattice, dims, tau, nranks=2, counts=None, faces=None, wall_u=None, storage="f32",
                 rho0=1.0, force=(0.0, 0.0, 0.0), tile=None, device=-1):
        self._lib = B.load()
        self.lattice = lattice
        lat_id = B.LATTICES[lattice] if isinstance(lattice, str) else int(lattice)
        self.d = 2 if lat_id == B.LB_D2Q9 else 3
        self.q = {0: 9, 1: 19, 2: 27}[lat_id]
        dims = list(dims) + [1] * (3 - len(dims))
        self.dims = tuple(int(v) for v in dims[:3])
        self.n = self.dims[0] * self.dims[1] * self.dims[2]
        bnd = B.lb_boundary()
        faces = faces if faces is not None else [B.LB_PERIODIC] * 6
        for k in range(6):
            fk = faces[k] if k < len(faces) else B.LB_PERIODIC
            bnd.kind[k] = Solver._FACE[fk] if isinstance(fk, str) else int(fk)
            for al in range(3):
                bnd.wall_u[k][al] = float(wall_u[k][al]) if wall_u is not None else 0.0
        opt = B.lb_options()
        self._lib.lb_default_options(ctypes.byref(opt))
        opt.storage = B.STORAGES[storage] if isinstance(storage, str) else int(storage)
        opt.rho0 = float(rho0)
        for k in range(3):
            opt.force[k] = float(force[k]) if k < len(force) else 0.0
        if tile is not None:
            for k in range(3):
                opt.tile[k] = int(tile[k]) if k < len(tile) else 0
        opt.device = int(device)
        cnt = (ctypes.c_int64 * nranks)(*counts) if counts is not None else None
        self._g = ctypes.c_void_p()
        B.check(self._lib.lb_group_create(lat_id, (ctypes.c_int64 * 3)(*self.dims), float(tau), ctypes.byref(bnd),
                                          ctypes.byref(opt), int(nranks), cnt, ctypes.byref(self._g)),
                "lb_group_create")
        slow = self.d - 1
        plane = self.n // self.dims[slow]  # nodes per plane of the slowest axis
        self.ranks, self.ranges = [], []
        for r in range(nranks):
            c = ctypes.c_void_p()
            off = ctypes.c_int64()
            B.check(self._lib.lb_group_rank(self._g, r, ctypes.byref(c), ctypes.byref(off)), "lb_group_rank")
            rd = list(self.dims)
            rd[slow] = (counts[r] if counts is not None else
                        self.dims[slow] // nranks + (1 if r < self.dims[slow] % nranks else 0))
            self.ranks.append(Solver._view(c.value, lattice, rd, rho0))
            self.ranges.append((off.value * plane, (off.value + rd[slow]) * plane))

    def _split(self, a, comps):
        a = np.asarray(a, dtype=np.float64).reshape(comps, self.n)
        return [np.ascontiguousarray(a[:, n0:n1]) for n0, n1 in self.ranges]

    def set_populations(self, f):
        for s, part in zip(self.ranks, self._split(f, self.q)):
            s.set_populations(part)

    def get_populations(self):
        return np.concatenate([s.get_populations() for s in self.ranks], axis=1)

    def init_moments(self, rho, u, pineq=None):
        np_ = 3 if self.d == 2 else 6
        rs, us = self._split(rho, 1), self._split(u, self.d)
        ps = self._split(pineq, np_) if pineq is not None else [None] * len(self.ranks)
        for s, r, uu, p in zip(self.ranks, rs, us, ps):
            s.init_moments(np.ascontiguousarray(r[0]), uu, p)

    def moments(self):
        parts = [s.moments() for s in self.ranks]
        return np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts], axis=1)

    def step(self, n=1):
        B.check(self._lib.lb_group_step(self._g, int(n)), "lb_group_step")

    def sync(self):
        B.check(self._lib.lb_group_sync(self._g), "lb_group_sync")

    def close(self):
        if getattr(self, "_g", None) and self._g.value:
            for s in self.ranks:
                s.close()
            self._lib.lb_group_destroy(self._g)
            self._g = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class CGSolver:
    """Two-component colour-gradient domain (lb_cg_*): periodic box, D2Q9 or
    D3Q19, storage "f64" or "f32"."""

    def __init__(self, lattice, dims, tau, sigma, beta, storage="f32", stream=None):
        self._lib = B.load()
        self.lat_id = B.LATTICES[lattice] if isinstance(lattice, str) else int(lattice)
        self.d = 2 if self.lat_id == B.LB_D2Q9 else 3
        self.q = 9 if self.lat_id == B.LB_D2Q9 else 19
        dims = list(dims) + [1] * (3 - len(dims))
        self.dims = tuple(int(v) for v in dims[:3])
        self.n = self.dims[0] * self.dims[1] * self.dims[2]
        self._c = ctypes.c_void_p()
        st = ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream))) if stream is not None else None
        B.check(self._lib.lb_cg_create(self.lat_id, (ctypes.c_int64 * 3)(*self.dims), float(tau), float(sigma),
                                       float(beta), B.STORAGES[storage] if isinstance(storage, str) else int(storage),
                                       st, ctypes.byref(self._c)), "lb_cg_create")

    def init(self, rho_r, rho_b, u=None):
        pr, dev = _ptr(rho_r)
        pb, dev2 = _ptr(rho_b)
        pu, dev3 = _ptr(u)
        if u is None:
            dev3 = dev
        if not (dev == dev2 == dev3):
            raise ValueError("rho_r, rho_b and u must all be host or all be device buffers")
        B.check(self._lib.lb_cg_init(self._c, pr, pb, pu, dev), "lb_cg_init")

    def set_populations(self, fr, fb):
        pr, dev = _ptr(fr)
        pb, dev2 = _ptr(fb)
        if dev != dev2:
            raise ValueError("f_r and f_b must both be host or both be device buffers")
        B.check(self._lib.lb_cg_set_populations(self._c, pr, pb, dev), "lb_cg_set_populations")

    def get_populations(self):
        fr, fb = np.empty((self.q, self.n)), np.empty((self.q, self.n))
        B.check(self._lib.lb_cg_get_populations(self._c, ctypes.c_void_p(fr.ctypes.data),
                                                ctypes.c_void_p(fb.ctypes.data), 0), "lb_cg_get_populations")
        return fr, fb

    def set_nci(self, amplitude, eps=0.1, h=1):
        """Near-contact interactions (section 2.2): repulsive force
        amplitude * rho_R * n on nodes flagged around thin films of the blue
        phase (bulk: phi < -1 + eps; sampling distance h); 0 switches off."""
        B.check(self._lib.lb_cg_set_nci(self._c, float(amplitude), float(eps), int(h)), "lb_cg_set_nci")

    def step(self, n=1):
        B.check(self._lib.lb_cg_step(self._c, int(n)), "lb_cg_step")

    def sync(self):
        B.check(self._lib.lb_cg_sync(self._c), "lb_cg_sync")

    def fields(self, rho_r=None, rho_b=None, u=None):
        """(rho_R, rho_B, u); pass torch CUDA tensors to stay on the device."""
        if rho_r is None and rho_b is None and u is None:
            rho_r, rho_b, u = np.empty(self.n), np.empty(self.n), np.empty((self.d, self.n))
        ptrs = [_ptr(x) for x in (rho_r, rho_b, u)]
        devs = {d for (p, d), x in zip(ptrs, (rho_r, rho_b, u)) if x is not None}
        if len(devs) != 1:
            raise ValueError("outputs must all be host or all be device buffers")
        B.check(self._lib.lb_cg_fields(self._c, ptrs[0][0], ptrs[1][0], ptrs[2][0], devs.pop()), "lb_cg_fields")
        return rho_r, rho_b, u

    def close(self):
        if getattr(self, "_c", None) and self._c.value:
            self._lib.lb_cg_destroy(self._c)
            self._c = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def lattice_table(lattice):
    lib = B.load()
    lid = B.LATTICES[lattice] if isinstance(lattice, str) else int(lattice)
    q = {0: 9, 1: 19, 2: 27}[lid]
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q)
    opp = np.zeros(q, dtype=np.int32)
    B.check(lib.lb_lattice_table(lid, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "lb_lattice_table")
    return c, w, opp


def fused_plan(lattice, dims, storage="f32", tile=None, sms=0) -> dict:
    """The brick decomposition lb_create() would choose (lb_plan_fused; no
    device is touched)."""
    lib = B.load()
    lid = B.LATTICES[lattice] if isinstance(lattice, str) else int(lattice)
    st = B.STORAGES[storage] if isinstance(storage, str) else int(storage)
    dims = list(dims) + [1] * (3 - len(dims))
    t = (ctypes.c_int32 * 3)(*tile) if tile is not None else None
    p = B.lb_plan_t()
    B.check(lib.lb_plan_fused(lid, st, (ctypes.c_int64 * 3)(*[int(v) for v in dims[:3]]), t, int(sms),
                              ctypes.byref(p)), "lb_plan_fused")
    return {name: getattr(p, name) for name, _ in p._fields_}


def memory_plan(lattice, bytes_per_value=4) -> dict:
    lib = B.load()
    lid = B.LATTICES[lattice] if isinstance(lattice, str) else int(lattice)
    p = B.lb_memory_plan_t()
    B.check(lib.lb_memory_plan(lid, int(bytes_per_value), ctypes.byref(p)), "lb_memory_plan")
    return {name: getattr(p, name) for name, _ in p._fields_}
