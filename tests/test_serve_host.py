"""Host logic of the continuous-batching server, without a GPU.

The solver and the batch are replaced by fakes whose residual falls by a fixed
factor per round, so admission order, the memory and node caps, retirement
and the report can be checked on the CPU.  The GPU tests check that served
results equal solo runs bit for bit.
"""
import numpy as np
import pytest

from paper_2304_06437_gb300 import serve


class FakeSolver:
    live = 0

    def __init__(self, lattice, dims, tau, faces=None, wall_u=None, force=(0, 0, 0), storage="f32", stream=None):
        self.n = int(np.prod(dims))
        self.steps = 0
        self.last = None
        self.rate = 0.5 if tau > 0.8 else 0.8  # residual factor per 100 steps
        FakeSolver.live += 1

    def step(self, n):
        self.steps += n

    def reduce(self, residual=False):
        r = 1.0 if self.last is None else self.rate ** (self.steps / 100.0)
        self.last = self.steps
        return {"mass": float(self.n), "momentum": [0.0, 0.0, 0.0], "residual": r}

    def moments(self):
        return np.ones(self.n), np.zeros((3, self.n))

    def close(self):
        FakeSolver.live -= 1


class FakeBatch:
    def __init__(self, solvers, stream=None):
        self.solvers = list(solvers)

    def step(self, n):
        for s in self.solvers:
            s.step(n)

    def reduce(self, residual=False):
        return [s.reduce(residual) for s in self.solvers]

    def sync(self):
        pass

    def close(self):
        pass


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(serve, "Solver", FakeSolver)
    monkeypatch.setattr(serve, "Batch", FakeBatch)
    FakeSolver.live = 0
    return serve


class Clock:
    def __init__(self, dt):
        self.t, self.dt = 0.0, dt

    def __call__(self):
        self.t += self.dt
        return self.t


def _req(rid, arrival, L, tau=0.9, tol=1e-3):
    return serve.Request(rid=rid, arrival=arrival, lattice="D3Q19", dims=(L, L, L), tau=tau, faces=[1] * 6, tol=tol)


def test_all_requests_finish_and_resources_are_freed(fake):
    srv = fake.Server(round_steps=100, clock=Clock(0.01), free_bytes=lambda: 1 << 40, reserve_bytes=0)
    reqs = [_req(i, 0.005 * i, 10 + i) for i in range(8)]
    for r in reqs:
        srv.submit(r)
    done = srv.run()
    assert len(done) == 8 and all(r.converged for r in done)
    assert FakeSolver.live == 0
    # residual 0.5**k < 1e-3 first at k = 10 rounds
    assert all(r.steps == 1000 for r in done)
    rep = srv.report(1.0)
    assert rep["completed"] == 8 and rep["latency_p50_s"] is not None


def test_node_cap_and_smallest_first(fake):
    srv = fake.Server(round_steps=100, clock=Clock(0.01), free_bytes=lambda: 1 << 40, reserve_bytes=0,
                      max_active_nodes=30 ** 3, order="smallest")
    sizes = [28, 12, 20, 14]
    reqs = [_req(i, 0.0, L) for i, L in enumerate(sizes)]
    for r in reqs:
        srv.submit(r)
    srv.step_round()
    admitted = sorted(r.rid for r, _ in srv.active)
    # smallest first (12, 14, 20) fits under 27000 nodes; 28^3 alone exceeds the rest
    assert admitted == [1, 2, 3]
    done = srv.run()
    assert len(done) == 4
    assert max(r.admitted for r in done if r.rid != 0) < next(r.admitted for r in done if r.rid == 0)


def test_step_cap_retires_unconverged(fake):
    srv = fake.Server(round_steps=100, clock=Clock(0.01), free_bytes=lambda: 1 << 40, reserve_bytes=0)
    r = _req(0, 0.0, 10, tau=0.6, tol=1e-12)
    r.max_steps = 500
    srv.submit(r)
    done = srv.run()
    assert done[0].steps == 500 and not done[0].converged
    assert srv.report(1.0)["capped_or_diverged"] == 1


def test_poisson_stream_is_seeded_and_in_range():
    a = serve.poisson_requests(50, 50.0, seed=1)
    b = serve.poisson_requests(50, 50.0, seed=1)
    assert [x.arrival for x in a] == [x.arrival for x in b]
    assert all(32 <= x.dims[0] <= 256 for x in a)
    assert all(x.tau >= 0.51 for x in a)
    assert np.all(np.diff([x.arrival for x in a]) > 0)


def test_allocation_failure_keeps_the_request_queued(fake, monkeypatch):
    """A request whose allocation fails while others are resident stays in
    the queue and is admitted after a resident domain retires."""
    from paper_2304_06437_gb300 import _binding as B

    class FailingOnce(FakeSolver):
        failed = False

        def __init__(self, lattice, dims, *a, **k):
            if dims[0] == 30 and not FailingOnce.failed:
                FailingOnce.failed = True
                raise B.LBError(B.LB_E_NOMEM, "lb_create")
            super().__init__(lattice, dims, *a, **k)

    monkeypatch.setattr(serve, "Solver", FailingOnce)
    srv = fake.Server(round_steps=100, clock=Clock(0.01), free_bytes=lambda: 1 << 40, reserve_bytes=0)
    srv.submit(_req(0, 0.0, 10))
    srv.submit(_req(1, 0.0, 30))
    srv.step_round()
    assert [r.rid for r, _ in srv.active] == [0] and [r.rid for r in srv.queue] == [1]
    done = srv.run()
    assert sorted(r.rid for r in done) == [0, 1] and all(r.converged for r in done)
    assert FakeSolver.live == 0


def test_allocation_failure_on_an_empty_server_is_raised(fake, monkeypatch):
    from paper_2304_06437_gb300 import _binding as B

    def failing(*a, **k):
        raise B.LBError(B.LB_E_NOMEM, "lb_create")

    monkeypatch.setattr(serve, "Solver", failing)
    srv = fake.Server(round_steps=100, clock=Clock(0.01), free_bytes=lambda: 1 << 40, reserve_bytes=0)
    srv.submit(_req(0, 0.0, 10))
    with pytest.raises(B.LBError):
        srv.step_round()
