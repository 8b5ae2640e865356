"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/lb.h declares, validates arguments before touching
the device, and its host tables agree with the independent oracle's."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2304_06437_gb300 import _binding as B
from paper_2304_06437_gb300 import build as lbbuild
from paper_2304_06437_gb300 import lattice_table, memory_plan

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    lbbuild.build()
    return B.load()


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "lb.h")).read()
    return sorted(set(re.findall(r"^LB_API\s+[\w\s\*]+?\b(lb_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_abi():
    names = _declared_symbols()
    for required in ["lb_create", "lb_step", "lb_moments", "lb_destroy", "lb_init_moments",
                     "lb_set_populations", "lb_get_populations", "lb_reduce", "lb_sync"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    names = _declared_symbols()
    assert set(names) == set(B.SIGNATURES), "binding and header disagree"
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    assert lib.lb_status_string(0) == b"ok"
    assert lib.lb_status_string(B.LB_E_TIMEOUT) == b"kernel wait timed out"
    assert lib.lb_abi_version() == 1


def test_create_rejects_bad_arguments_without_a_device(lib):
    ctx = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 3)(8, 8, 8)
    opt = B.lb_options()
    lib.lb_default_options(ctypes.byref(opt))
    assert lib.lb_create(7, dims, 0.8, None, ctypes.byref(opt), ctypes.byref(ctx)) == B.LB_E_INVAL
    assert lib.lb_create(B.LB_D3Q19, dims, 0.5, None, ctypes.byref(opt), ctypes.byref(ctx)) == B.LB_E_INVAL
    d2 = (ctypes.c_int64 * 3)(8, 8, 2)
    assert lib.lb_create(B.LB_D2Q9, d2, 0.8, None, ctypes.byref(opt), ctypes.byref(ctx)) == B.LB_E_INVAL
    bad = B.lb_boundary()
    bad.kind[0] = B.LB_WALL  # -x wall with periodic +x
    assert lib.lb_create(B.LB_D3Q19, dims, 0.8, ctypes.byref(bad), ctypes.byref(opt), ctypes.byref(ctx)) == B.LB_E_INVAL
    opt.storage = 9
    assert lib.lb_create(B.LB_D3Q19, dims, 0.8, None, ctypes.byref(opt), ctypes.byref(ctx)) == B.LB_E_INVAL
    assert lib.lb_step(None, 1) == B.LB_E_INVAL
    assert lib.lb_sync(None) == B.LB_E_INVAL


def test_slab_calls_reject_bad_arguments_without_a_device(lib):
    ctx = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 3)(8, 8, 8)
    opt = B.lb_options()
    lib.lb_default_options(ctypes.byref(opt))
    link_x = B.lb_boundary()
    link_x.kind[0] = link_x.kind[1] = B.LB_LINK  # link faces only on the slowest axis
    assert lib.lb_create(B.LB_D3Q19, dims, 0.8, ctypes.byref(link_x), ctypes.byref(opt), ctypes.byref(ctx)) == \
        B.LB_E_INVAL
    link_z = B.lb_boundary()
    link_z.kind[4] = link_z.kind[5] = B.LB_LINK
    bad_kind = B.lb_boundary()
    bad_kind.kind[4] = bad_kind.kind[5] = 4
    assert lib.lb_create(B.LB_D3Q19, dims, 0.8, ctypes.byref(bad_kind), ctypes.byref(opt), ctypes.byref(ctx)) == \
        B.LB_E_INVAL
    opt.scheme = B.LB_SCHEME_TWO_PASS
    assert lib.lb_create(B.LB_D3Q19, dims, 0.8, ctypes.byref(link_z), ctypes.byref(opt), ctypes.byref(ctx)) == \
        B.LB_E_UNSUPPORTED
    lib.lb_default_options(ctypes.byref(opt))
    grp = ctypes.c_void_p()
    # a group places the links itself; counts must cover the slowest axis
    assert lib.lb_group_create(B.LB_D3Q19, dims, 0.8, ctypes.byref(link_z), ctypes.byref(opt), 2, None,
                               ctypes.byref(grp)) == B.LB_E_INVAL
    assert lib.lb_group_create(B.LB_D3Q19, dims, 0.8, None, ctypes.byref(opt), 9, None, ctypes.byref(grp)) == \
        B.LB_E_INVAL
    assert lib.lb_group_create(B.LB_D3Q19, dims, 0.8, None, ctypes.byref(opt), 2, (ctypes.c_int64 * 2)(3, 4),
                               ctypes.byref(grp)) == B.LB_E_INVAL
    assert lib.lb_group_create(B.LB_D3Q19, dims, 0.8, None, ctypes.byref(opt), 2, (ctypes.c_int64 * 2)(8, 0),
                               ctypes.byref(grp)) == B.LB_E_INVAL
    opt.scheme = B.LB_SCHEME_TWO_PASS
    assert lib.lb_group_create(B.LB_D3Q19, dims, 0.8, None, ctypes.byref(opt), 2, None, ctypes.byref(grp)) == \
        B.LB_E_UNSUPPORTED
    n = ctypes.c_int64()
    assert lib.lb_halo_bytes(None, ctypes.byref(n)) == B.LB_E_INVAL
    assert lib.lb_halo_pack(None, 0, None) == B.LB_E_INVAL
    assert lib.lb_halo_unpack(None, 1, None) == B.LB_E_INVAL
    assert lib.lb_group_step(None, 1) == B.LB_E_INVAL
    assert lib.lb_group_sync(None) == B.LB_E_INVAL
    assert lib.lb_group_rank(None, 0, None, None) == B.LB_E_INVAL
    lib.lb_group_destroy(None)


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19", "D3Q27"])
def test_lattice_table_matches_oracle(lat):
    c, w, opp = lattice_table(lat)
    co, wo, oppo = oracle.lattice_tables(lat)
    assert (c == co).all()
    assert np.abs(w - wo).max() == 0.0
    assert (opp == oppo).all()


def test_memory_plan_matches_paper_counts():
    """Section 4: 15 vs 21 arrays in 2D (D2Q9), 29 vs 42 in 3D (D3Q19);
    24 and 52 bytes saved per node in single precision."""
    import json
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "memory_accounting.json")))
    for lat, row in gold["lattices"].items():
        p = memory_plan(lat, 4)
        assert p["arrays_moment_scheme"] == row["arrays_thread_safe"]
        assert p["arrays_flip_flop"] == row["arrays_flip_flop"]
        saved = p["bytes_per_node_flip_flop"] - p["bytes_per_node_moment_scheme"]
        assert saved == row["bytes_saved_per_node_fp32"]
        # and the fused single-array scheme keeps q arrays only
        assert p["arrays_single"] == p["q"]
    # 1e9 nodes in 3D: about 50 GB saved by the moment scheme
    p = memory_plan("D3Q19", 4)
    saved_gb = (p["bytes_per_node_flip_flop"] - p["bytes_per_node_moment_scheme"]) * 1e9 / 1e9
    assert abs(saved_gb - gold["saving_at_1e9_nodes_gb"]) < 3
