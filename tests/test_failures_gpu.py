"""Failure detection without a GPU fault.

Errors are made on the host or in data, and the one kernel-side failure (a
wait that never completes) is a bounded wait on a barrier that nothing
completes: the kernel records LB_E_TIMEOUT and returns, the context stays
usable.  Nothing here traps, faults or hangs a GPU."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import torch
    assert torch.cuda.is_available()
    from paper_2304_06437_gb300 import build
    build.build()
    import paper_2304_06437_gb300 as P
    from paper_2304_06437_gb300 import _binding as B
    return P, B


def test_bounded_wait_times_out_and_device_stays_usable(lb):
    P, B = lb
    lib = B.load()
    waited = ctypes.c_int64()
    rc = lib.lb_selftest_timeout(200_000_000, ctypes.byref(waited))  # 0.2 s
    assert rc == B.LB_E_TIMEOUT
    assert 0.2e9 <= waited.value < 2.0e9
    # the context is still healthy: a normal solve afterwards
    with P.Solver("D3Q19", (16, 12, 10), 0.7) as s:
        s.step(3)
        s.sync()
        r = s.reduce()
    assert abs(r["mass"] - 16 * 12 * 10) < 1e-9


def test_allocation_failure_reports_nomem(lb):
    P, B = lb
    with pytest.raises(P.LBError) as e:
        P.Solver("D3Q19", (1 << 14, 1 << 14, 1 << 10), 0.7)  # ~2e13 bytes: cudaMalloc refuses
    assert e.value.code == B.LB_E_NOMEM


def test_non_finite_state_reports_diverged(lb):
    P, B = lb
    from lbcase import random_state
    dims = (20, 9, 7)
    f = np.ascontiguousarray(random_state("D3Q19", dims, 3))
    f[4, 17] = np.nan  # a host-made fault in the data
    with P.Solver("D3Q19", dims, 0.7, storage="f32") as s:
        s.set_populations(f)
        s.step(2)
        with pytest.raises(P.LBError) as e:
            s.reduce(residual=True)
        assert e.value.code == B.LB_E_DIVERGED


def test_bad_arguments_are_rejected_before_gpu_work(lb):
    P, B = lb
    for args in [("D3Q19", (0, 4, 4), 0.7), ("D3Q19", (4, 4, 4), 0.5), ("D2Q9", (4, 4, 3), 0.7)]:
        with pytest.raises(P.LBError) as e:
            P.Solver(*args)
        assert e.value.code == B.LB_E_INVAL
