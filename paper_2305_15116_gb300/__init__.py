"""GB300-native matrix-free P1 operator apply on block-structured meshes.

A thin Python binding over libhyteg.so (C ABI in include/hyteg.h).  The
library implements the apply of Thönnes & Rüde (PASC '23): an unstructured
coarse mesh of triangles or tetrahedra, every macro refined uniformly to level
L, and y = A x with constant per-macro stencils plus an interface step
(Sec. 1.2, Sec. 5).  PyTorch provides device memory and streams only.
"""
from .mesh import (Mesh, F64, F32, F64_IEEE, BC_NONE, BC_DIRICHLET, SOLVE_F64, SOLVE_MIXED, HytegError,
                   version, apply_batch, solve_two_part_group)
from .server import Server, Result
from ._capi import REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED

__all__ = ["Mesh", "F64", "F32", "F64_IEEE", "BC_NONE", "BC_DIRICHLET", "SOLVE_F64", "SOLVE_MIXED", "HytegError",
           "version", "apply_batch", "solve_two_part_group", "Server", "Result", "REQ_QUEUED", "REQ_RUNNING", "REQ_DONE", "REQ_FAILED"]
