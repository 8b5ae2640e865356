"""Continuous-batching solve server on one GPU.

Requests (one lattice Boltzmann solve each: lattice, cube side, boundaries,
tau, force, storage, a convergence threshold and a step cap) arrive over
time.  The engine keeps every admitted domain resident in device memory and
advances all of them together, ``round_steps`` time steps per round, through
one :class:`~paper_2304_06437_gb300.solver.Batch` (one persistent launch per
brick-shape class and step, CUDA-graph replays).  Between rounds it

* reads every active domain's FP64 relative velocity residual
  ||u_t - u_{t-K}|| / ||u_t|| (K = round_steps) in one batched reduction
  (``lb_batch_reduce``: one pass per domain on the device, one copy to the
  host) and retires the domains that converged or hit their step cap (their
  rho and u are copied to the host and their device memory freed);
* admits arrived requests (first come first served, or smallest first) while
  the device's free memory minus a reserve covers the request's estimated
  footprint and an optional cap on resident nodes allows, so requests that
  arrive while others run join the next round;
* rebuilds the batch when its membership changed.

Every domain takes whole rounds from its own admission, so its step count
and its convergence decision depend on its own state only: each result is
bit for bit the one of solving the request alone with the same round length
(the batch is bitwise equal to solo stepping).

Only argument marshalling and bookkeeping happen here; every step runs in
the CUDA library.
"""
from __future__ import annotations

import dataclasses
import math
import time
from typing import Callable, List, Optional

import numpy as np

from ._binding import LB_E_NOMEM, LBError
from .solver import Batch, Solver


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float                 # seconds on the server clock
    lattice: str
    dims: tuple
    tau: float
    faces: list
    wall_u: Optional[list] = None
    force: tuple = (0.0, 0.0, 0.0)
    storage: str = "f32"
    tol: float = 1e-6              # relative velocity residual over one round
    max_steps: int = 200000
    # filled in by the server
    admitted: float = float("nan")
    finished: float = float("nan")
    steps: int = 0
    residual: float = float("nan")
    converged: bool = False
    rho: Optional[np.ndarray] = None
    u: Optional[np.ndarray] = None


Q_OF = {"D2Q9": 9, "D3Q19": 19, "D3Q27": 27}
BYTES_OF = {"f64": 8, "f32": 4, "f16s": 2, "bf16s": 2}


def footprint_bytes(req: Request) -> int:
    """Device bytes a request holds while resident: the population array,
    the brick shells (bounded by a quarter of the populations for the
    compiled brick shapes), the FP32 residual snapshot of u and slack."""
    n = int(np.prod(req.dims))
    pop = Q_OF[req.lattice] * BYTES_OF[req.storage] * n
    return int(1.25 * pop + 12 * n + (4 << 20))


class Server:
    """Continuous batching over a request stream.

    clock: returns the server time in seconds (default: wall time since
    start).  keep_fields: copy rho and u of finished requests to the host.
    """

    def __init__(self, round_steps: int = 100, reserve_bytes: int = 2 << 30, clock: Optional[Callable[[], float]] = None,
                 free_bytes: Optional[Callable[[], int]] = None, keep_fields: bool = True, stream=None,
                 max_active_nodes: Optional[int] = None, order: str = "fifo"):
        import torch
        self.torch = torch
        self.round_steps = int(round_steps)
        self.reserve = int(reserve_bytes)
        t0 = time.perf_counter()
        self.clock = clock or (lambda: time.perf_counter() - t0)
        self.free_bytes = free_bytes or (lambda: torch.cuda.mem_get_info()[0])
        self.keep_fields = keep_fields
        self.stream = stream
        # admission policy: a cap on resident nodes keeps rounds short under
        # overload; "smallest" admits the smallest arrived request first
        # (shortest-job-first by size), "fifo" in arrival order
        self.max_active_nodes = max_active_nodes
        if order not in ("fifo", "smallest"):
            raise ValueError("order must be 'fifo' or 'smallest'")
        self.order = order
        self.queue: List[Request] = []
        self.active: List[tuple] = []       # (request, solver)
        self.done: List[Request] = []
        self.batch: Optional[Batch] = None
        self.updates = 0                    # node updates executed
        self.rounds = 0
        self.max_active = 0
        # host wall time per phase of the rounds (seconds)
        self.phase_s = {"admit": 0.0, "rebuild": 0.0, "step": 0.0, "retire": 0.0}

    # ---------------------------------------------------------------- engine
    def submit(self, req: Request):
        self.queue.append(req)

    def _admit(self) -> bool:
        changed = False
        now = self.clock()
        while True:
            arrived = [i for i, r in enumerate(self.queue) if r.arrival <= now]
            if not arrived:
                break
            if self.order == "smallest":
                pick = min(arrived, key=lambda i: (int(np.prod(self.queue[i].dims)), self.queue[i].arrival))
            else:
                pick = arrived[0]
            req = self.queue[pick]
            need = footprint_bytes(req)
            if self.active and self.free_bytes() - need < self.reserve:
                break  # wait for memory; an empty server always admits
            if (self.active and self.max_active_nodes is not None and
                    sum(s.n for _, s in self.active) + int(np.prod(req.dims)) > self.max_active_nodes):
                break
            try:
                s = Solver(req.lattice, req.dims, req.tau, faces=req.faces, wall_u=req.wall_u, force=req.force,
                           storage=req.storage, stream=self.stream)
            except LBError as e:
                # the footprint estimate fell short, or another process took
                # the memory since it was read: keep the request queued and
                # retry once a resident domain retires (an empty server has
                # nothing to wait for, so there the error stands)
                if e.code != LB_E_NOMEM or not self.active:
                    raise
                break
            self.queue.pop(pick)
            s.reduce(residual=True)  # residual baseline: u at admission
            req.admitted = self.clock()
            self.active.append((req, s))
            changed = True
        return changed

    def _retire(self) -> bool:
        keep, changed = [], False
        # the batch's members are the active domains, in this order
        sums = self.batch.reduce(residual=True)
        for (req, s), red in zip(self.active, sums):
            r = red["residual"]
            req.residual = r
            if not math.isfinite(r) or r < req.tol or req.steps >= req.max_steps:
                req.converged = math.isfinite(r) and r < req.tol
                if self.keep_fields:
                    req.rho, req.u = s.moments()
                s.close()
                req.finished = self.clock()
                self.done.append(req)
                changed = True
            else:
                keep.append((req, s))
        self.active = keep
        return changed

    def _rebuild(self):
        if self.batch is not None:
            self.batch.close()
            self.batch = None
        if self.active:
            self.batch = Batch([s for _, s in self.active], stream=self.stream)

    def step_round(self):
        """One round: admit, advance every active domain by round_steps,
        retire converged ones."""
        t0 = time.perf_counter()
        changed = self._admit()
        t1 = time.perf_counter()
        if changed or (self.batch is None and self.active):
            self._rebuild()
        t2 = time.perf_counter()
        self.phase_s["admit"] += t1 - t0
        self.phase_s["rebuild"] += t2 - t1
        self.max_active = max(self.max_active, len(self.active))
        if not self.active:
            return
        self.batch.step(self.round_steps)
        self.batch.sync()
        t3 = time.perf_counter()
        for req, s in self.active:
            req.steps += self.round_steps
            self.updates += s.n * self.round_steps
        self.rounds += 1
        retired = self._retire()
        t4 = time.perf_counter()
        if retired:
            self._rebuild()
        self.phase_s["step"] += t3 - t2
        self.phase_s["retire"] += t4 - t3
        self.phase_s["rebuild"] += time.perf_counter() - t4

    def run(self, until: Optional[float] = None, idle_sleep: float = 1e-3):
        """Serve until the queue and the engine are empty (or the clock passes
        `until`; requests still queued or active are then left unfinished)."""
        while self.queue or self.active:
            if until is not None and self.clock() >= until:
                break
            if not self.active and self.queue and self.queue[0].arrival > self.clock():
                time.sleep(min(idle_sleep, max(0.0, self.queue[0].arrival - self.clock())))
                continue
            self.step_round()
        return self.done

    def close(self):
        if self.batch is not None:
            self.batch.close()
            self.batch = None
        for _, s in self.active:
            s.close()
        self.active = []

    # ---------------------------------------------------------------- report
    def report(self, wall_s: float) -> dict:
        lat = np.array([r.finished - r.arrival for r in self.done]) if self.done else np.zeros(0)
        gpu = np.array([r.finished - r.admitted for r in self.done]) if self.done else np.zeros(0)

        def pct(a, p):
            return float(np.percentile(a, p)) if a.size else None

        return {
            "completed": len(self.done), "converged": int(sum(r.converged for r in self.done)),
            "capped_or_diverged": int(sum(not r.converged for r in self.done)),
            "queued_unserved": len(self.queue), "active_unfinished": len(self.active),
            "latency_p50_s": pct(lat, 50), "latency_p99_s": pct(lat, 99),
            "on_gpu_p50_s": pct(gpu, 50), "on_gpu_p99_s": pct(gpu, 99),
            "aggregate_mlups": self.updates / wall_s / 1e6 if wall_s > 0 else None,
            "rounds": self.rounds, "max_active": self.max_active,
            "host_phase_s": {k: round(v, 3) for k, v in self.phase_s.items()},
        }


def solve_alone(req: Request, round_steps: int, stream=None):
    """Reference: the request solved by itself with the server's round length
    and convergence rule (same steps, same decision, same bits)."""
    s = Solver(req.lattice, req.dims, req.tau, faces=req.faces, wall_u=req.wall_u, force=req.force,
               storage=req.storage, stream=stream)
    s.reduce(residual=True)
    steps = 0
    while True:
        s.step(round_steps)
        steps += round_steps
        r = s.reduce(residual=True)["residual"]
        if not math.isfinite(r) or r < req.tol or steps >= req.max_steps:
            break
    f = s.get_populations()
    rho, u = s.moments()
    s.close()
    return steps, r, f, rho, u


def poisson_requests(n: int, rate: float, seed: int, side_range=(32, 256), re_range=(10.0, 1000.0),
                     lid_u: float = 0.05, tau_min: float = 0.51, storages=("f32", "f16s"), tol: float = 1e-6,
                     max_steps: int = 200000) -> List[Request]:
    """Seeded D3Q19 cavity / duct stream: Poisson arrivals, cube sides and
    Reynolds numbers log-uniform, tau = 1/2 + 3 U L / Re (U = lid speed, or the
    duct's centre-line target); where tau would fall below tau_min it is held
    there and U lowered to keep Re.  The duct is driven by the body force
    that gives the target centre-line speed of a square duct."""
    g = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(n):
        t += g.exponential(1.0 / rate)
        L = int(round(math.exp(g.uniform(math.log(side_range[0]), math.log(side_range[1])))))
        Re = float(math.exp(g.uniform(math.log(re_range[0]), math.log(re_range[1]))))
        U = lid_u
        tau = 0.5 + 3.0 * U * L / Re
        if tau < tau_min:
            tau = tau_min
            U = (tau - 0.5) * Re / (3.0 * L)
        storage = storages[int(g.integers(0, len(storages)))]
        if i % 2 == 0:
            faces = [1, 1, 1, 2, 1, 1]
            wall_u = [[0, 0, 0]] * 3 + [[U, 0, 0]] + [[0, 0, 0]] * 2
            force = (0.0, 0.0, 0.0)
        else:
            # square duct along x, walls at +-y and +-z; the centre-line speed of
            # a square duct is about 0.0737 F L^2 / (rho0 nu)
            faces = [0, 0, 1, 1, 1, 1]
            wall_u = None
            nu = (tau - 0.5) / 3.0
            force = (U * nu / (0.0737 * L * L), 0.0, 0.0)
        out.append(Request(rid=i, arrival=t, lattice="D3Q19", dims=(L, L, L), tau=tau, faces=faces, wall_u=wall_u,
                           force=force, storage=storage, tol=tol, max_steps=max_steps))
    return out
