"""GB300-native thread-safe regularized lattice Boltzmann (arXiv 2304.06437).

The compute path is the CUDA library in ``csrc/`` (C ABI: include/lb.h),
built for sm_103a by :mod:`paper_2304_06437_gb300.build`.  This package only
binds it; there is no CPU fallback.
"""
from ._binding import LBError, load  # noqa: F401
from .solver import Batch, CGSolver, SlabGroup, Solver, fused_plan, lattice_table, memory_plan  # noqa: F401

__all__ = ["Solver", "Batch", "CGSolver", "SlabGroup", "LBError", "fused_plan", "lattice_table", "memory_plan",
           "load"]
