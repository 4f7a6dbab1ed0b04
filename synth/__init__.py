"""Seeded synthetic inputs for the two-strip list-mode MLEM workloads.

This package is shared by the FP64 oracle tests and by the CUDA path's tests and
benchmarks.  It holds only input generation: phantoms (ellipse tables in the
layout of the paper's App. A table) and simulated detector events (the measured
triple of Sec. 2: hit positions z_u, z_d along the two strips and the path-length
difference delta_l).  It contains none of the reconstruction arithmetic (no direct
reconstruction, no kernel, no sensitivity, no MLEM update).
"""
from .phantom import Ellipse, Phantom, paper_phantom, random_phantom
from .events import Geometry, simulate_events
from .configs import WORKLOADS, Workload, batched_instances, make_workload

__all__ = [
    "Ellipse", "Phantom", "paper_phantom", "random_phantom",
    "Geometry", "simulate_events",
    "WORKLOADS", "Workload", "batched_instances", "make_workload",
]
