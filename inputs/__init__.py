"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds no arithmetic of the method itself: it only builds coarse
meshes (vertex coordinates and cell connectivity) and draws random vectors from
seeds.  Both the CPU oracle and the CUDA path consume what it produces; neither
depends on the other.
"""
from .meshes import (
    CoarseMesh,
    unit_square_mesh,
    unit_cube_kuhn_mesh,
    rect_mesh,
    box_kuhn_mesh,
    random_vector,
    range_vector,
    random_normal,
    workload,
    WORKLOADS,
)

__all__ = [
    "CoarseMesh",
    "unit_square_mesh",
    "unit_cube_kuhn_mesh",
    "rect_mesh",
    "box_kuhn_mesh",
    "random_vector",
    "range_vector",
    "random_normal",
    "workload",
    "WORKLOADS",
]
