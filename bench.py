#!/usr/bin/env python3
"""Throughput of the fused single-array regularized lattice Boltzmann step.

Metric: MLUPS (million lattice-node updates per second, the paper's GLUPS x
1e3) on one GB300, with the dominant kernel's fraction of the HBM roofline.
Default workload: D3Q19 lid-driven cavity, 1024^3 nodes (one FP32 population
array, 81.6 GB), tau = 0.52, lid velocity 0.05, started from rest.

A step is one time step over the whole grid (one launch of the fused kernel).
The grid (81.6 GB) is far larger than L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the workload
(replicas only: the single-domain step has no multi-GPU path here) and rank 0
prints the whole-job rate.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import shutil
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: lattice, dims, tau, boundary kind, parameters
    "cavity_d3q19_1024": dict(lattice="D3Q19", dims=(1024, 1024, 1024), tau=0.52, flow="cavity", lid=0.05),
    "cavity_d3q19_512": dict(lattice="D3Q19", dims=(512, 512, 512), tau=0.52, flow="cavity", lid=0.05),
    "cavity_d3q19_256": dict(lattice="D3Q19", dims=(256, 256, 256), tau=0.52, flow="cavity", lid=0.05),
    # the 1024^3 cavity cut into two z-slabs, each a context with its own
    # stream, halos exchanged on the device between steps (the slab
    # decomposition of a two-GPU run, emulated on one GPU)
    "cavity_d3q19_1024_slabs2": dict(lattice="D3Q19", dims=(1024, 1024, 1024), tau=0.52, flow="cavity", lid=0.05,
                                     slabs=2),
    # profiling case: 2.5 GB, yet every brick sweeps 512 planes as at 1024^3
    "cavity_d3q19_256x512": dict(lattice="D3Q19", dims=(256, 256, 512), tau=0.52, flow="cavity", lid=0.05),
    # the D3Q27 Taylor-Green vortex at 1.07e9 nodes (one FP32 array, 116 GB)
    "tg_d3q27_1024": dict(lattice="D3Q27", dims=(1024, 1024, 1024), tau=0.8, flow="tg3d", u0=0.02),
    "tg_d3q27_512": dict(lattice="D3Q27", dims=(512, 512, 512), tau=0.8, flow="tg3d", u0=0.02),
    "tg_d3q27_256": dict(lattice="D3Q27", dims=(256, 256, 256), tau=0.8, flow="tg3d", u0=0.02),
    "tg_d2q9_16384": dict(lattice="D2Q9", dims=(16384, 16384, 1), tau=0.8, flow="tg2d", u0=0.01),
    # force-driven channel (walls at +-y, periodic x and z) started from the
    # analytic parabola; the force 1e-6 of an H = 64 channel is scaled by
    # (64/512)^2 so that the peak velocity stays 0.0154 at H = 512
    "channel_d3q27_512": dict(lattice="D3Q27", dims=(512, 512, 512), tau=0.6, flow="channel",
                              force=1e-6 * (64.0 / 512.0) ** 2),
    "channel_d3q27_64": dict(lattice="D3Q27", dims=(64, 64, 64), tau=0.6, flow="channel", force=1e-6),
    # 256 independent domains in one batch: 128 D2Q9 squares (side log-uniform
    # 32..1024) and 128 D3Q19 cubes (16..128), tau uniform in [0.55, 1.2], per
    # lattice half Taylor-Green (periodic) and half lid-driven cavity, FP32
    "batch_256": dict(lattice="mixed", dims=None, tau=None, flow="batch", n2d=128, n3d=128),
    # continuous batching: Poisson arrivals (50 / s) of D3Q19 cavity and duct
    # solves, cubes 32..256, Re 10..1000, FP32 or shifted-FP16 storage, each run
    # until the relative velocity residual over 100 steps is below 1e-6 (cap
    # 2e5 steps), served for a fixed wall-clock horizon
    "serve_d3q19": dict(lattice="D3Q19", dims=None, tau=None, flow="serve", n_req=200, rate=50.0),
    # two-component colour-gradient model: an emulsion of seeded droplets in a
    # periodic box (the paper's two-component sizes: 4096^2 and 256^3)
    "cg_d2q9_4096": dict(lattice="D2Q9", dims=(4096, 4096, 1), tau=1.0, flow="cg", sigma=0.01, beta=0.7,
                         drops=2000, radius=(8, 24)),
    "cg_d3q19_256": dict(lattice="D3Q19", dims=(256, 256, 256), tau=1.0, flow="cg", sigma=0.01, beta=0.7,
                         drops=300, radius=(6, 16)),
    # the same 2D emulsion with near-contact interactions (section 2.2):
    # amplitude 0.01, bulk threshold eps = 0.1, sampling distance h = 2
    "cg_d2q9_4096_nci": dict(lattice="D2Q9", dims=(4096, 4096, 1), tau=1.0, flow="cg", sigma=0.01, beta=0.7,
                             drops=2000, radius=(8, 24), nci=(0.01, 0.1, 2)),
}
Q = {"D2Q9": 9, "D3Q19": 19, "D3Q27": 27}
STORAGE_BYTES = {"f64": 8, "f32": 4, "f16s": 2, "bf16s": 2}


def boundary(w):
    if w["flow"] == "cavity":
        faces = [1, 1, 1, 2, 1, 1]
        wall_u = [[0, 0, 0]] * 3 + [[w["lid"], 0, 0]] + [[0, 0, 0]] * 2
        return faces, wall_u
    if w["flow"] == "channel":
        return [0, 0, 1, 1, 0, 0], None
    return [0] * 6, None


def force_of(w):
    return (w.get("force", 0.0), 0.0, 0.0)


def channel_fields(w, torch):
    """Analytic Poiseuille profile u_x(y) = F/(2 rho0 nu) (y + 1/2)(H - 1/2 - y)
    (walls half a link outside nodes 0 and H - 1), built on the device."""
    nx, ny, nz = w["dims"]
    nu = (w["tau"] - 0.5) / 3.0
    y = torch.arange(ny, device="cuda", dtype=torch.float64)
    prof = w["force"] / (2.0 * nu) * (y + 0.5) * (ny - 0.5 - y)
    return prof


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def read_traffic(kernel_key):
    """DRAM bytes per node update measured by ncu (profiles/*.txt), or None."""
    p = os.path.join(ROOT, "profiles", "traffic_per_update.txt")
    try:
        for line in open(p):
            line = line.strip()
            if line.startswith(kernel_key + " "):
                return float(line.split()[1])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        exe = shutil.which("nvidia-smi")
        if not exe:
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.fh = open(self.path, "w")
        self.proc = subprocess.Popen([exe, "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                      "-i", str(self.dev), "-lms", "200"], stdout=self.fh,
                                     stderr=subprocess.DEVNULL)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x, torch):
    """The largest value over the ranks of the default process group (the
    value itself without one): the job's time is its slowest rank's."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, torch):
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_state(solver, w, torch):
    """Synthetic initial condition, generated on the device."""
    if w["flow"] == "cavity":
        solver.init_uniform(1.0, (0.0, 0.0, 0.0))
        return
    import synth
    if w["flow"] == "channel":
        nx, ny, nz = w["dims"]
        N = nx * ny * nz
        rho = torch.ones(N, device="cuda", dtype=torch.float64)
        u = torch.zeros((3, N), device="cuda", dtype=torch.float64)
        u[0].view(nz, ny, nx).copy_(channel_fields(w, torch).view(1, ny, 1).expand(nz, ny, nx))
        solver.init_moments(rho, u)
        del rho, u
        torch.cuda.empty_cache()
        return
    if w["flow"] == "tg3d":
        rho, u, pi = synth.taylor_green_3d_torch(w["dims"][0], w["u0"], 1.0, w["tau"], torch)
    else:
        rho, u, pi = synth.taylor_green_2d_torch(w["dims"][0], w["u0"], 1.0, w["tau"], torch)
    solver.init_moments(rho, u, pi)
    del rho, u, pi
    torch.cuda.empty_cache()


def run_reference(args, w):
    """--impl reference: the CPU oracle, timed on a bounded sample of the
    workload (the sample of the default run's cpu_baseline: the workload's
    flow at its parity size)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    lattice = w["lattice"]
    dims, _ = PARITY_SIZE[w["flow"]]
    wsz = dict(w)
    wsz["dims"] = dims
    if w["flow"] == "channel":
        wsz["force"] = 1e-6
    faces, wall_u = boundary(wsz)
    if lattice == "D2Q9":
        faces = faces[:4] + [0, 0]
    cfg = oracle.make_cfg(lattice, dims, w["tau"], force=force_of(wsz), faces=faces, wall_u=wall_u)
    rho, u, pineq = parity_fields(wsz, dims)
    f = oracle.init(cfg, rho, u, pineq)
    f = oracle.run(cfg, f, args.warmup)
    t0 = time.perf_counter()
    f = oracle.run(cfg, f, args.steps)
    dt = time.perf_counter() - t0
    N = dims[0] * dims[1] * dims[2]
    value = N * args.steps / dt / 1e6
    cores = oracle.max_threads()
    sample = "%s %s %s, %d timed steps (FP64 CPU oracle, two arrays, OpenMP)" % (
        lattice, w["flow"], "x".join(map(str, dims)), args.steps)
    line = {
        "impl": "reference", "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "sample": sample},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cavity_d3q19_1024", choices=sorted(WORKLOADS))
    ap.add_argument("--storage", default="f32", choices=sorted(STORAGE_BYTES))
    ap.add_argument("--scheme", default="fused", choices=["fused", "two_pass"])
    ap.add_argument("--tile", default=None, help="bx,by,bz")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="serving horizon (serve workload)")
    ap.add_argument("--serve-max-nodes", type=int, default=1 << 26, help="cap on resident nodes (serve workload)")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, w)
        return
    if w["flow"] == "batch":
        run_batch(args, w)
        return
    if w["flow"] == "serve":
        run_serve(args, w)
        return
    if w["flow"] == "cg":
        run_cg(args, w)
        return
    if w.get("slabs"):
        run_slabs(args, w)
        return

    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2304_06437_gb300 import Solver

    lattice, dims, tau = w["lattice"], w["dims"], w["tau"]
    faces, wall_u = boundary(w)
    N = dims[0] * dims[1] * dims[2]
    stream = torch.cuda.Stream()
    tile = tuple(int(v) for v in args.tile.split(",")) if args.tile else None
    s = Solver(lattice, dims, tau, faces=faces, wall_u=wall_u, storage=args.storage, scheme=args.scheme,
               stream=stream, tile=tile, force=force_of(w))
    info = s.info()
    init_state(s, w, torch)
    for _ in range(args.warmup):
        s.step(1)
    s.sync()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # ---- device-resident timing: events around every launch on the solver's stream
    clocks = ClockSampler(torch.cuda.current_device())
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev[0].record(stream)
    for i in range(args.steps):
        s.step(1)
        ev[i + 1].record(stream)
    s.sync()
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    per_launch = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = max_over_ranks(ev[0].elapsed_time(ev[args.steps]), torch)
    value = ws * N * args.steps / (total_ms * 1e-3) / 1e6
    ms_per_step = total_ms / args.steps
    launches_per_step = 1 if args.scheme == "fused" else 2

    es = STORAGE_BYTES[args.storage]
    q = Q[lattice]
    alg_bytes = 2 * q * es * N  # one read + one write of every population
    avg_launch_s = float(np.mean(per_launch)) * 1e-3
    peak, peak_kind = read_peaks()
    achieved = alg_bytes / avg_launch_s / 1e9
    # ncu bytes of the default brick shape: not for a requested brick or pipeline
    default_shape = args.tile is None and not os.environ.get("LB_FUSED_PIPELINE")
    traffic_per_update = read_traffic("%s_%s_%s" % (args.scheme, lattice, args.storage)) if default_shape else None
    roofline = {
        "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
        "peak_kind": peak_kind,
        "traffic": traffic_per_update * N if traffic_per_update else None,
        "kernel": "k1_fused_step" if args.scheme == "fused" else "k0_moments+k0_rebuild",
        "algorithmic_bytes_per_update": 2 * q * es,
    }

    # ---- accuracy of the timed run against the analytic profile (channel)
    accuracy = {}
    if w["flow"] == "channel":
        accuracy["u_vs_parabola_after_timed_steps"] = channel_error(s, w, torch)

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(s, w, args, torch, stream)

    s.close()
    # ---- CPU baseline (the FP64 oracle on a bounded sample) and, from the
    # same oracle run, the error of the benchmark's storage at a parity size
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu, ref = cpu_baseline_leg(w)
        if not args.no_accuracy:
            accuracy.update(side_accuracy(w, args, torch, ref))

    if rank == 0:
        line = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.storage == "f64" else "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "lattice": lattice, "dims": list(dims), "tau": tau,
                       "storage": args.storage, "scheme": args.scheme, "tile": list(info["tile"]),
                       "flow": w["flow"], "l2_flush": "inputs larger than L2 (%.1f GB population array)" % (
                           info["population_bytes"] / 1e9),
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "accuracy": accuracy,
            "gpu_launches": launches_per_step * args.steps,
            "per_launch_ms": {"mean": float(np.mean(per_launch)), "min": float(np.min(per_launch)),
                              "max": float(np.max(per_launch))},
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_slabs(args, w):
    """The single-domain workload as a slab group on one GPU (one context and
    stream per slab, halo messages between steps).  Timed by the host clock
    around synchronised steps (the ranks run on the group's own streams); the
    rate counts the whole domain's node updates."""
    import torch
    from paper_2304_06437_gb300 import SlabGroup
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    lattice, dims, tau = w["lattice"], w["dims"], w["tau"]
    faces, wall_u = boundary(w)
    N = dims[0] * dims[1] * dims[2]
    g = SlabGroup(lattice, dims, tau, nranks=w["slabs"], faces=faces, wall_u=wall_u, storage=args.storage,
                  force=force_of(w))
    g.step(args.warmup)
    g.sync()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    t0 = time.perf_counter()
    g.step(args.steps)
    g.sync()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    clk = clocks.stop()
    info = g.ranks[0].info()
    g.close()
    es = STORAGE_BYTES[args.storage]
    q = Q[lattice]
    peak, peak_kind = read_peaks()
    achieved = 2 * q * es * N * args.steps / dt / 1e9
    if rank == 0:
        line = {
            "metric": "MLUPS", "value": N * args.steps / dt / 1e6, "unit": "MLUPS", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.storage == "f64" else "f32", "data": "synthetic",
            "config": {"workload": args.workload, "lattice": lattice, "dims": list(dims), "tau": tau,
                       "storage": args.storage, "slabs": w["slabs"], "tile": list(info["tile"]),
                       "timing": "host clock around synchronised steps",
                       "l2_flush": "inputs larger than L2", "parallelism": "slab group on one GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "traffic": None, "kernel": "k1_fused_step (LINK) per slab",
                         "algorithmic_bytes_per_update": 2 * q * es},
            "cpu_baseline": None, "e2e": None, "clocks": clk,
            "gpu_launches": args.steps * w["slabs"] * 3,
        }
        print(json.dumps(line), flush=True)


def batch_specs(w, seed=20230412):
    """Domain list of the batching workload (seeded)."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for lat, n, lo, hi, u0 in (("D2Q9", w["n2d"], 32, 1024, 0.01), ("D3Q19", w["n3d"], 16, 128, 0.02)):
        for i in range(n):
            L = int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))
            tau = float(g.uniform(0.55, 1.2))
            flow = "tg" if i < n // 2 else "cavity"
            out.append(dict(lattice=lat, L=L, tau=tau, flow=flow, u0=u0))
    return out


def make_batch_domain(spec, storage, torch, stream=None):
    from paper_2304_06437_gb300 import Solver
    import synth
    lat, L, tau = spec["lattice"], spec["L"], spec["tau"]
    d = 2 if lat == "D2Q9" else 3
    dims = (L, L) if d == 2 else (L, L, L)
    if spec["flow"] == "cavity":
        faces = [1, 1, 1, 2, 1, 1] if d == 3 else [1, 1, 1, 2, 0, 0]
        wall_u = [[0, 0, 0]] * 3 + [[0.05, 0, 0]] + [[0, 0, 0]] * 2
        s = Solver(lat, dims, tau, faces=faces, wall_u=wall_u, storage=storage, stream=stream)
        s.init_uniform(1.0)
        return s
    s = Solver(lat, dims, tau, storage=storage, stream=stream)
    if d == 3:
        rho, u, pi = synth.taylor_green_3d_torch(L, spec["u0"], 1.0, tau, torch)
    else:
        rho, u, pi = synth.taylor_green_2d_torch(L, spec["u0"], 1.0, tau, torch)
    s.init_moments(rho, u, pi)
    return s


def run_batch(args, w):
    """Batching workload: all domains advance together, one persistent launch
    per brick-shape class and step, two steps per CUDA-graph replay; compared
    with the same domains stepped one after another with the single-domain
    kernel (one launch per domain and step)."""
    import torch
    from paper_2304_06437_gb300 import Batch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    specs = batch_specs(w)
    stream = torch.cuda.Stream()
    doms = [make_batch_domain(sp, args.storage, torch, stream) for sp in specs]
    torch.cuda.synchronize()
    N = sum(d.n for d in doms)
    q_of = {"D2Q9": 9, "D3Q19": 19, "D3Q27": 27}
    es = STORAGE_BYTES[args.storage]
    alg_bytes = sum(2 * q_of[sp["lattice"]] * es * d.n for sp, d in zip(specs, doms))
    # the same domains one after another with their own plans, one
    # single-domain launch per domain and step (measured before the batch
    # re-plans its members for batched throughput)
    seq_steps = max(2, min(args.steps, 20))
    for d in doms:
        d.step(1)
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(seq_steps):
        for d in doms:
            d.step(1)
    s1.record(stream)
    torch.cuda.synchronize()
    seq_ms = s0.elapsed_time(s1) / seq_steps
    seq_value = N / (seq_ms * 1e-3) / 1e6

    b = Batch(doms, stream=stream)
    info = b.info()
    b.step(args.warmup)
    b.sync()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    clocks = ClockSampler(torch.cuda.current_device())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0.record(stream)
    b.step(args.steps)
    e1.record(stream)
    b.sync()
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    total_ms = max_over_ranks(e0.elapsed_time(e1), torch)
    value = ws * N * args.steps / (total_ms * 1e-3) / 1e6
    b.close()
    for d in doms:
        d.close()
    peak, peak_kind = read_peaks()
    achieved = alg_bytes / (total_ms / args.steps * 1e-3) / 1e9
    if rank == 0:
        line = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "domains": len(specs), "nodes": N, "storage": args.storage,
                       "classes": info["n_classes"], "persistent_ctas": info["ctas"],
                       "work_items": info["work_items"], "graph": "2 steps per replay",
                       "l2_flush": "none: %.1f GB of populations per step, larger than L2" % (alg_bytes / 2e9),
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "traffic": None, "kernel": "k2_batched_step (all classes)",
                         "algorithmic_bytes_per_step": alg_bytes},
            "sequential_baseline": {"value": seq_value, "unit": "MLUPS", "ms_per_step": seq_ms,
                                    "what": "same domains, one single-domain launch per domain and step"},
            "cpu_baseline": None, "e2e": None, "clocks": clk,
            "gpu_launches": info["launches_per_step"] * args.steps,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_serve(args, w):
    """Serving workload: the request stream is replayed in real time against
    the continuous-batching server for --serve-seconds; reports latency
    percentiles of the requests that finished, the aggregate update rate and
    the offered versus served load."""
    import torch
    from paper_2304_06437_gb300 import serve
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    reqs = serve.poisson_requests(w["n_req"], w["rate"], seed=20230412 + rank)
    offered = sum(int(np.prod(r.dims)) for r in reqs)
    srv = serve.Server(round_steps=100, keep_fields=False, max_active_nodes=args.serve_max_nodes, order="smallest")
    for r in reqs:
        srv.submit(r)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    t0 = time.perf_counter()
    srv.run(until=args.serve_seconds)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    rep = srv.report(wall)
    srv.close()
    rate = sum_over_ranks(srv.updates / wall, torch) / 1e6
    if rank == 0:
        line = {
            "metric": "MLUPS", "value": rate, "unit": "MLUPS", "n_gpus": ws, "steps": srv.rounds * 100,
            "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "requests": len(reqs), "rate_per_s": w["rate"],
                       "horizon_s": args.serve_seconds, "round_steps": 100, "tol": 1e-6, "step_cap": 200000,
                       "admission": "smallest first, free HBM, at most %d resident nodes" % args.serve_max_nodes,
                       "offered_nodes": offered, "parallelism": "replicas" if ws > 1 else "single GPU"},
            "serving": rep, "roofline": None, "cpu_baseline": None, "e2e": None, "clocks": clk,
            "gpu_launches": None,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def emulsion_fields(w, torch, seed=20230412, device="cuda"):
    """Seeded droplets (red) in a blue matrix: phi = max over drops of
    tanh((R_i - r_i) / 2), built on the device one drop at a time."""
    g = np.random.Generator(np.random.PCG64(seed))
    nx, ny, nz = w["dims"]
    d = 2 if nz == 1 else 3
    N = nx * ny * nz
    phi = torch.full((nz, ny, nx), -1.0, device=device, dtype=torch.float64)
    ax = [torch.arange(n, device=device, dtype=torch.float64) for n in (nx, ny, nz)]
    for _ in range(w["drops"]):
        c = [g.uniform(0, n) for n in (nx, ny, nz)]
        R = g.uniform(*w["radius"])
        # periodic distances along each axis, only inside the drop's bounding box
        lo = [int(math.floor(ci - R - 4)) for ci in c]
        hi = [int(math.ceil(ci + R + 4)) for ci in c]
        idx = [torch.arange(l, h, device=device) % n for l, h, n in zip(lo, hi, (nx, ny, nz))]
        dd = [torch.remainder(ax[k][idx[k]] - c[k] + ax[k].numel() / 2, ax[k].numel()) - ax[k].numel() / 2
              for k in range(3)]
        if d == 2:
            r = torch.sqrt(dd[0].view(1, 1, -1) ** 2 + dd[1].view(1, -1, 1) ** 2)
            sub = phi[0:1][:, idx[1]][:, :, idx[0]]
            val = torch.maximum(sub, torch.tanh((R - r) / 2.0))
            phi[0:1, idx[1].view(-1, 1), idx[0].view(1, -1)] = val[0]
        else:
            r = torch.sqrt(dd[0].view(1, 1, -1) ** 2 + dd[1].view(1, -1, 1) ** 2 + dd[2].view(-1, 1, 1) ** 2)
            sub = phi[idx[2]][:, idx[1]][:, :, idx[0]]
            val = torch.maximum(sub, torch.tanh((R - r) / 2.0))
            phi[idx[2].view(-1, 1, 1), idx[1].view(1, -1, 1), idx[0].view(1, 1, -1)] = val
    phi = phi.reshape(N)
    return ((1 + phi) / 2).contiguous(), ((1 - phi) / 2).contiguous()


def run_cg(args, w):
    """Two-component colour-gradient workload: one step is the three launches
    (moments, phase-field gradient, rebuild of both colours)."""
    import torch
    from paper_2304_06437_gb300 import CGSolver
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    lattice, dims = w["lattice"], w["dims"]
    N = dims[0] * dims[1] * dims[2]
    q = Q[lattice]
    es = STORAGE_BYTES[args.storage]
    stream = torch.cuda.Stream()
    s = CGSolver(lattice, dims[:2] if dims[2] == 1 else dims, w["tau"], w["sigma"], w["beta"], storage=args.storage,
                 stream=stream)
    if "nci" in w:
        s.set_nci(*w["nci"])
    rr, rb = emulsion_fields(w, torch)
    s.init(rr, rb)
    del rr, rb
    torch.cuda.empty_cache()
    s.step(args.warmup)
    s.sync()
    clocks = ClockSampler(torch.cuda.current_device())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0.record(stream)
    s.step(args.steps)
    e1.record(stream)
    s.sync()
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = max_over_ranks(e0.elapsed_time(e1), torch)
    # mass of each colour is conserved: a cheap whole-run check
    R, B, _ = s.fields()
    s.close()
    value = ws * N * args.steps / (total_ms * 1e-3) / 1e6
    # algorithmic bytes of the three-launch schedule: both colours read and
    # written once (4 q s), 13 moment fields written and read back (26 r),
    # the phase field read and 4 gradient fields written and read (9 r)
    rs = 8 if args.storage == "f64" else 4
    alg = 4 * q * es + 35 * rs
    achieved = alg * N / (total_ms / args.steps * 1e-3) / 1e9
    peak, peak_kind = read_peaks()
    if rank == 0:
        line = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.storage == "f64" else "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "lattice": lattice, "dims": list(dims), "tau": w["tau"],
                       "sigma": w["sigma"], "beta": w["beta"], "drops": w["drops"], "storage": args.storage,
                       "nci": (dict(zip(("amplitude", "eps", "h"), w["nci"])) if "nci" in w else None),
                       "launches_per_step": 3, "l2_flush": "inputs larger than L2",
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind, "traffic": None,
                         "kernel": "cg_moments + cg_gradient + cg_rebuild", "algorithmic_bytes_per_update": alg},
            "mass": {"red": float(R.sum()), "blue": float(B.sum())},
            "cpu_baseline": None, "e2e": None, "clocks": clk, "gpu_launches": 3 * args.steps,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def channel_error(s, w, torch):
    """Relative L2 error of u (all nodes, all components) against the analytic
    channel profile, in FP64 on the device."""
    nx, ny, nz = w["dims"]
    N = nx * ny * nz
    rho = torch.empty(N, device="cuda", dtype=torch.float64)
    u = torch.empty((3, N), device="cuda", dtype=torch.float64)
    s.moments(rho, u)
    prof = channel_fields(w, torch).view(1, ny, 1)
    ux = u[0].view(nz, ny, nx)
    num = ((ux - prof) ** 2).sum() + (u[1] ** 2).sum() + (u[2] ** 2).sum()
    den = (prof.expand(nz, ny, nx) ** 2).sum()
    out = float(torch.sqrt(num / den))
    del rho, u
    torch.cuda.empty_cache()
    return out


PARITY_SIZE = {"cavity": ((64, 64, 64), 200), "tg3d": ((64, 64, 64), 200), "tg2d": ((256, 256, 1), 1000),
               "channel": ((64, 64, 64), 2000)}


def parity_fields(w, dims):
    """Initial (rho, u, pineq) of the workload's flow at a parity size, as
    host arrays (the same seeded/analytic fields feed the oracle and the GPU)."""
    import synth
    d = 2 if w["lattice"] == "D2Q9" else 3
    if w["flow"] == "cavity":
        rho, u = synth.rest_state(dims, d)
        return rho, u, None
    if w["flow"] == "channel":
        rho, u = synth.channel_state(dims, 1e-6, 1.0, (w["tau"] - 0.5) / 3.0, d)
        return rho, u, None
    if w["flow"] == "tg3d":
        return synth.taylor_green_3d(dims[0], w["u0"], 1.0, w["tau"])
    return synth.taylor_green_2d(dims[0], w["u0"], 1.0, w["tau"])


def cpu_baseline_leg(w, budget_s=12.0, threads=0):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the workload:
    the workload's flow at its parity size (cavity and Taylor-Green 64^3 x 200
    steps, 2D Taylor-Green 256^2 x 1000, channel from the parabola 2000
    steps), timed on the host cores.  Its final rho and u are also the FP64
    reference of the benchmark's accuracy field.  If the parity run takes less
    than the budget, the sample continues from its end state until the budget
    is spent, and the rate covers every timed step.  (The channel flow is
    uniform in x and z, so its reference runs on a 1 x 64 x 1 column, whose
    fields equal every column of the 64^3 box; the timing runs the 64^3 box.)"""
    import oracle
    dims, steps = PARITY_SIZE[w["flow"]]
    ws = dict(w)
    ws["dims"] = dims
    if w["flow"] == "channel":
        ws["force"] = 1e-6  # the H = 64 force of the channel study
    faces, wall_u = boundary(ws)
    lattice = w["lattice"]
    if lattice == "D2Q9":
        faces = faces[:4] + [0, 0]
    rdims = (1, dims[1], 1) if w["flow"] == "channel" else dims
    rcfg = oracle.make_cfg(lattice, rdims, w["tau"], force=force_of(ws), faces=faces, wall_u=wall_u)
    rho, u, pineq = parity_fields(ws, rdims)
    f = oracle.init(rcfg, rho, u, pineq)
    t0 = time.perf_counter()
    f = oracle.run(rcfg, f, steps, threads)
    dt_ref = time.perf_counter() - t0
    ref = oracle.moments(rcfg, f)
    # timing sample: the parity run itself, extended on the full parity box
    if w["flow"] == "channel":
        tcfg = oracle.make_cfg(lattice, dims, w["tau"], force=force_of(ws), faces=faces, wall_u=wall_u)
        rho, u, pineq = parity_fields(ws, dims)
        ft = oracle.init(tcfg, rho, u, pineq)
        timed_updates, dt = 0, 0.0
    else:
        tcfg, ft = rcfg, f
        timed_updates, dt = dims[0] * dims[1] * dims[2] * steps, dt_ref
    N = dims[0] * dims[1] * dims[2]
    extra = 0
    while dt < budget_s:
        t0 = time.perf_counter()
        ft = oracle.run(tcfg, ft, 10, threads)
        dt += time.perf_counter() - t0
        timed_updates += N * 10
        extra += 10
    used = threads if threads > 0 else oracle.max_threads()
    sample = "%s %s %s, %d timed steps (FP64 oracle, two arrays, OpenMP); its %d-step state is the accuracy " \
             "reference" % (lattice, w["flow"], "x".join(map(str, dims)), timed_updates // N, steps)
    cpu = {"value": timed_updates / dt / 1e6, "unit": "MLUPS", "cores": used, "kind": "oracle", "sample": sample}
    return cpu, ref


def side_accuracy(w, args, torch, ref):
    """The benchmark's storage and scheme at the parity size of its flow, from
    the same initial fields as the oracle run of the CPU-baseline leg, against
    that FP64 oracle result: relative L2 of rho, rho - rho0 and u."""
    from paper_2304_06437_gb300 import Solver
    dims, steps = PARITY_SIZE[w["flow"]]
    ws = dict(w)
    ws["dims"] = dims
    if w["flow"] == "channel":
        ws["force"] = 1e-6
    faces, wall_u = boundary(ws)
    s = Solver(w["lattice"], dims, w["tau"], faces=faces, wall_u=wall_u, storage=args.storage,
               scheme=args.scheme, force=force_of(ws))
    rho0, u0, pi0 = parity_fields(ws, dims)
    s.init_moments(rho0, np.ascontiguousarray(u0), None if pi0 is None else np.ascontiguousarray(pi0))
    s.step(steps)
    rho, u = s.moments()
    s.close()
    r_ref, u_ref = ref
    if w["flow"] == "channel":  # the column's fields, repeated over x and z
        nx, ny, nz = dims
        r_ref = np.broadcast_to(r_ref.reshape(1, ny, 1), (nz, ny, nx)).reshape(-1)
        u_ref = np.broadcast_to(u_ref.reshape(-1, 1, ny, 1), (u_ref.shape[0], nz, ny, nx)).reshape(u_ref.shape[0], -1)

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    return {"vs": "FP64 CPU oracle", "size": "x".join(map(str, dims)), "steps": steps,
            "rho_rel_l2": rel(rho, r_ref), "drho_rel_l2": rel(rho - 1.0, r_ref - 1.0) if np.any(r_ref != 1.0)
            else None, "u_rel_l2": rel(u, u_ref)}


def measure_e2e(s, w, args, torch, stream):
    """Same metric through the public API with pinned host buffers: host
    (rho, u) -> lb_init_moments -> K steps -> lb_moments -> host."""
    dims = w["dims"]
    N = dims[0] * dims[1] * dims[2]
    d = 2 if w["lattice"] == "D2Q9" else 3
    try:
        rho_h = torch.empty(N, dtype=torch.float64, pin_memory=True)
        u_h = torch.empty((d, N), dtype=torch.float64, pin_memory=True)
        rho_o = torch.empty(N, dtype=torch.float64, pin_memory=True)
        u_o = torch.empty((d, N), dtype=torch.float64, pin_memory=True)
    except Exception as exc:  # host memory too small for the full workload
        return {"value": None, "unit": "MLUPS", "error": "pinned allocation failed: %s" % str(exc)[:120]}
    rho_h.fill_(1.0)
    u_h.zero_()
    rn, un, ro, uo = (t.numpy() for t in (rho_h, u_h, rho_o, u_o))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.init_moments(rn, un)
    s.step(args.steps)
    s.moments(ro, uo)
    dt = time.perf_counter() - t0
    h2d = (1 + d) * N * 8
    return {"value": N * args.steps / dt / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": h2d / args.steps,
            "d2h_bytes_per_step": h2d / args.steps, "seconds": dt}


if __name__ == "__main__":
    main()
