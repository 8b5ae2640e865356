"""Continuous-batching server (paper_2304_06437_gb300.serve).

Requests arrive over (virtual) time while others are on the GPU; they are
admitted between rounds as memory allows and stepped together in one batch.
Each request's result must equal solving it alone with the same round length
and convergence rule (bit for bit: the batch is bitwise equal to solo
stepping and the convergence decision depends on the request's own state).
Admission under a memory limit must delay, not drop, requests.  Each served
result is also compared with the FP64 CPU oracle run from the same rest state
for the same number of steps: relative L2 of rho and u within 1e-5 for FP32
storage.  FP16 storage is held to 5e-2 on u, a gate that catches a wrong
result, not the rounding error: in a weakly driven duct (u ~ 1e-3, body force
~1e-6 per step) the storage's quantum of the shifted populations is close to
the per-step force increment, and the steady state drifts by about 1 %
(measured 1.3e-2 on a 14^3 duct).
"""
import numpy as np
import pytest

import oracle
from lbcase import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import torch
    assert torch.cuda.is_available()
    from paper_2304_06437_gb300 import build
    build.build()
    import paper_2304_06437_gb300 as P
    from paper_2304_06437_gb300 import serve
    return P, serve


class StepClock:
    """Virtual clock: advances by a fixed amount per call, so that arrivals
    interleave with rounds deterministically."""

    def __init__(self, dt):
        self.t = 0.0
        self.dt = dt

    def __call__(self):
        self.t += self.dt
        return self.t


def _stream(serve, n, seed):
    reqs = serve.poisson_requests(n, rate=50.0, seed=seed, side_range=(10, 20), re_range=(5.0, 60.0),
                                  tol=1e-5, max_steps=3000)
    return reqs


def test_served_results_equal_solo(lb):
    P, serve = lb
    reqs = _stream(serve, 10, seed=3)
    srv = serve.Server(round_steps=50, clock=StepClock(0.01), reserve_bytes=0)
    for r in reqs:
        srv.submit(r)
    done = srv.run()
    srv.close()
    assert len(done) == len(reqs)
    assert srv.max_active >= 3  # requests overlapped on the device
    # later arrivals were admitted while earlier ones were still running
    assert any(a.admitted < b.finished and b.admitted < a.finished for a in done for b in done if a is not b)
    for r in done:
        steps, res, f, rho, u = serve.solve_alone(r, 50)
        assert r.steps == steps
        assert r.residual == res
        assert np.array_equal(r.rho, rho) and np.array_equal(r.u, u)
    # the served results against the oracle (rest start, same step count)
    for r in done:
        cfg = oracle.make_cfg(r.lattice, r.dims, r.tau, force=r.force, faces=r.faces, wall_u=r.wall_u)
        n = int(np.prod(r.dims))
        # lb_create's state: every population at its rest value t_a rho0
        f0 = np.repeat(oracle.lattice_tables(r.lattice)[1][:, None], n, axis=1)
        r_ref, u_ref = oracle.moments(cfg, oracle.run(cfg, f0, r.steps))
        tol_u = 1e-5 if r.storage == "f32" else 5e-2
        assert rel_l2(r.rho, r_ref) < (1e-5 if r.storage == "f32" else 1e-3)
        assert rel_l2(r.u, u_ref) < tol_u, (r.rid, r.storage, rel_l2(r.u, u_ref))


def test_admission_waits_for_memory(lb):
    P, serve = lb
    reqs = _stream(serve, 6, seed=5)
    foot = [serve.footprint_bytes(r) for r in reqs]
    budget = max(foot) * 2  # room for about two requests at a time
    holder = {}

    seen = []

    def free_bytes():
        held = sum(serve.footprint_bytes(r) for r, _ in holder["srv"].active)
        seen.append(held)
        return budget - held

    srv = serve.Server(round_steps=50, clock=StepClock(0.05), reserve_bytes=0, free_bytes=free_bytes)
    holder["srv"] = srv
    for r in reqs:
        srv.submit(r)
    done = srv.run()
    srv.close()
    assert len(done) == len(reqs)            # nothing dropped
    assert max(seen) <= budget               # never above the memory budget
    assert srv.max_active < len(reqs)        # some requests had to wait
    assert all(r.admitted >= r.arrival for r in done)
