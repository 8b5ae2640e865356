"""ctypes mirror of include/lb.h (argument marshalling only).

Every entry point of the C ABI is bound here under its own name.  Loading
fails loudly if the compiled library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbgb.so")

LB_OK = 0
LB_E_INVAL = -1
LB_E_NOMEM = -2
LB_E_CUDA = -3
LB_E_DIVERGED = -4
LB_E_TIMEOUT = -5
LB_E_UNSUPPORTED = -6
LB_E_TOO_LARGE = -7
LB_E_ABANDONED = -8
LB_NOALLOC_SCRATCH_BYTES = 64 << 20

LB_D2Q9, LB_D3Q19, LB_D3Q27 = 0, 1, 2
LB_PERIODIC, LB_WALL, LB_MOVING_WALL, LB_LINK = 0, 1, 2, 3
LB_F64, LB_F32, LB_F16S, LB_BF16S = 0, 1, 2, 3
LB_SCHEME_FUSED, LB_SCHEME_TWO_PASS = 0, 1

LATTICES = {"D2Q9": LB_D2Q9, "D3Q19": LB_D3Q19, "D3Q27": LB_D3Q27}
STORAGES = {"f64": LB_F64, "f32": LB_F32, "f16s": LB_F16S, "bf16s": LB_BF16S}
SCHEMES = {"fused": LB_SCHEME_FUSED, "two_pass": LB_SCHEME_TWO_PASS}


class lb_boundary(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32 * 6), ("wall_u", (ctypes.c_double * 3) * 6)]


class lb_options(ctypes.Structure):
    _fields_ = [
        ("storage", ctypes.c_int32),
        ("scheme", ctypes.c_int32),
        ("rho0", ctypes.c_double),
        ("force", ctypes.c_double * 3),
        ("stream", ctypes.c_void_p),
        ("tile", ctypes.c_int32 * 3),
        ("device", ctypes.c_int32),
    ]


class lb_info_t(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int32),
        ("q", ctypes.c_int32),
        ("d", ctypes.c_int32),
        ("storage", ctypes.c_int32),
        ("scheme", ctypes.c_int32),
        ("dims", ctypes.c_int64 * 3),
        ("steps_done", ctypes.c_int64),
        ("tile", ctypes.c_int32 * 3),
        ("population_bytes", ctypes.c_uint64),
        ("aux_bytes", ctypes.c_uint64),
        ("algorithmic_bytes_per_update", ctypes.c_uint64),
        ("nodes_per_thread", ctypes.c_int32),
        ("tma_slots", ctypes.c_int32),
    ]


class lb_memory_plan_t(ctypes.Structure):
    _fields_ = [
        ("q", ctypes.c_int32),
        ("m", ctypes.c_int32),
        ("arrays_moment_scheme", ctypes.c_int32),
        ("arrays_flip_flop", ctypes.c_int32),
        ("arrays_single", ctypes.c_int32),
        ("bytes_per_node_moment_scheme", ctypes.c_double),
        ("bytes_per_node_flip_flop", ctypes.c_double),
        ("bytes_per_node_single", ctypes.c_double),
    ]


class lb_tune_entry(ctypes.Structure):
    _fields_ = [
        ("bx", ctypes.c_int32),
        ("by", ctypes.c_int32),
        ("bz", ctypes.c_int32),
        ("slots", ctypes.c_int32),
        ("nodes_per_thread", ctypes.c_int32),
        ("export_warps", ctypes.c_int32),
        ("status", ctypes.c_int32),
        ("ns_per_update", ctypes.c_double),
    ]


class lb_plan_t(ctypes.Structure):
    _fields_ = [("bx", ctypes.c_int32), ("by", ctypes.c_int32), ("bz", ctypes.c_int32),
                ("nbx", ctypes.c_int32), ("nby", ctypes.c_int32), ("nbz", ctypes.c_int32),
                ("bricks", ctypes.c_int64), ("tma_slots", ctypes.c_int32), ("nodes_per_thread", ctypes.c_int32),
                ("export_warps", ctypes.c_int32), ("shared_bytes", ctypes.c_int64),
                ("shell_elems_per_parity", ctypes.c_int64)]


class lb_batch_info_t(ctypes.Structure):
    _fields_ = [
        ("n_domains", ctypes.c_int32),
        ("n_classes", ctypes.c_int32),
        ("launches_per_step", ctypes.c_int32),
        ("ctas", ctypes.c_int32),
        ("work_items", ctypes.c_int64),
        ("total_nodes", ctypes.c_int64),
        ("steps_done", ctypes.c_int64),
    ]


class LBError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (what, status_string(code), code))


_P = ctypes.POINTER
_vp = ctypes.c_void_p
_i64p = _P(ctypes.c_int64)
_dp = _P(ctypes.c_double)

# name -> (restype, argtypes); one line per declaration of include/lb.h
SIGNATURES = {
    "lb_default_options": (None, [_P(lb_options)]),
    "lb_create": (ctypes.c_int, [ctypes.c_int32, _i64p, ctypes.c_double, _P(lb_boundary), _P(lb_options), _P(_vp)]),
    "lb_init_moments": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int32]),
    "lb_init_uniform": (ctypes.c_int, [_vp, ctypes.c_double, _dp]),
    "lb_set_populations": (ctypes.c_int, [_vp, _vp, ctypes.c_int32]),
    "lb_get_populations": (ctypes.c_int, [_vp, _vp, ctypes.c_int32]),
    "lb_get_region": (ctypes.c_int, [_vp, _i64p, _i64p, _vp]),
    "lb_step": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "lb_moments": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32]),
    "lb_reduce": (ctypes.c_int, [_vp, _dp, _dp, _dp]),
    "lb_sync": (ctypes.c_int, [_vp]),
    "lb_destroy": (None, [_vp]),
    "lb_info": (ctypes.c_int, [_vp, _P(lb_info_t)]),
    "lb_lattice_table": (ctypes.c_int, [ctypes.c_int32, _P(ctypes.c_int32), _dp, _P(ctypes.c_int32)]),
    "lb_memory_plan": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _P(lb_memory_plan_t)]),
    "lb_step_noalloc": (ctypes.c_int, [ctypes.c_int32, _i64p, ctypes.c_double, _P(lb_boundary), ctypes.c_double,
                                       _dp, _vp, ctypes.c_int64, _vp]),
    "lb_autotune": (ctypes.c_int, [_vp, ctypes.c_int32, _P(lb_tune_entry), ctypes.c_int32, _P(ctypes.c_int32)]),
    "lb_batch_create": (ctypes.c_int, [_P(_vp), ctypes.c_int32, _vp, _P(_vp)]),
    "lb_batch_step": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "lb_batch_sync": (ctypes.c_int, [_vp]),
    "lb_batch_info": (ctypes.c_int, [_vp, _P(lb_batch_info_t)]),
    "lb_batch_reduce": (ctypes.c_int, [_vp, ctypes.c_int32, _dp]),
    "lb_batch_destroy": (None, [_vp]),
    "lb_cg_create": (ctypes.c_int, [ctypes.c_int32, _i64p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int32, _vp, _P(_vp)]),
    "lb_cg_init": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int32]),
    "lb_cg_set_populations": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32]),
    "lb_cg_get_populations": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32]),
    "lb_cg_step": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "lb_cg_fields": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int32]),
    "lb_cg_sync": (ctypes.c_int, [_vp]),
    "lb_cg_destroy": (None, [_vp]),
    "lb_cg_set_nci": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_int32]),
    "lb_plan_fused": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _i64p, _P(ctypes.c_int32), ctypes.c_int32,
                                     _P(lb_plan_t)]),
    "lb_halo_bytes": (ctypes.c_int, [_vp, _i64p]),
    "lb_halo_pack": (ctypes.c_int, [_vp, ctypes.c_int32, _vp]),
    "lb_halo_unpack": (ctypes.c_int, [_vp, ctypes.c_int32, _vp]),
    "lb_group_create": (ctypes.c_int, [ctypes.c_int32, _i64p, ctypes.c_double, _P(lb_boundary), _P(lb_options),
                                       ctypes.c_int32, _i64p, _P(_vp)]),
    "lb_group_rank": (ctypes.c_int, [_vp, ctypes.c_int32, _P(_vp), _i64p]),
    "lb_group_step": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "lb_group_sync": (ctypes.c_int, [_vp]),
    "lb_group_destroy": (None, [_vp]),
    "lb_selftest_timeout": (ctypes.c_int, [ctypes.c_int64, _i64p]),
    "lb_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "lb_abi_version": (ctypes.c_int, []),
}

_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load the compiled library (build it first with paper_2304_06437_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(
                "the CUDA library %s is not built; run `python -m paper_2304_06437_gb300.build` "
                "(this package has no CPU fallback)" % p)
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def status_string(code: int) -> str:
    try:
        return load().lb_status_string(int(code)).decode()
    except Exception:
        return "status %d" % code


def check(code: int, what: str) -> int:
    if code < 0:
        raise LBError(code, what)
    return code
