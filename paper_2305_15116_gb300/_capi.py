"""ctypes declarations of libhyteg.so (the C ABI of include/hyteg.h).

Argument marshalling only: every step of the operator runs in the library.
Importing this module fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhyteg.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"libhyteg.so not found at {LIB_PATH}; build it with "
        "`python paper_2305_15116_gb300/build.py` (nvcc, sm_103a)")

lib = ctypes.CDLL(LIB_PATH)

c_i64p = ctypes.POINTER(ctypes.c_int64)
c_dblp = ctypes.POINTER(ctypes.c_double)

lib.hyteg_mesh_create.argtypes = [ctypes.c_int, ctypes.c_int64, c_dblp, ctypes.c_int64, c_i64p, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_void_p)]
lib.hyteg_mesh_create.restype = ctypes.c_int
lib.hyteg_mesh_refine.argtypes = [ctypes.c_void_p, ctypes.c_int]
lib.hyteg_mesh_refine.restype = ctypes.c_int
lib.hyteg_mesh_destroy.argtypes = [ctypes.c_void_p]
lib.hyteg_mesh_destroy.restype = None
lib.hyteg_num_slots.argtypes = [ctypes.c_void_p, ctypes.c_int, c_i64p, c_i64p]
lib.hyteg_num_slots.restype = ctypes.c_int
lib.hyteg_dof_map.argtypes = [ctypes.c_void_p, ctypes.c_int, c_i64p]
lib.hyteg_dof_map.restype = ctypes.c_int
lib.hyteg_apply.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                            ctypes.c_void_p]
lib.hyteg_apply.restype = ctypes.c_int
lib.hyteg_apply_timed.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
lib.hyteg_apply_timed.restype = ctypes.c_int
lib.hyteg_apply_host.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p]
lib.hyteg_apply_host.restype = ctypes.c_int
lib.hyteg_apply_host_static.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]
lib.hyteg_apply_host_static.restype = ctypes.c_int
lib.hyteg_slot_coords.argtypes = [ctypes.c_void_p, ctypes.c_int, c_dblp]
lib.hyteg_slot_coords.restype = ctypes.c_int
lib.hyteg_lumped_mass.argtypes = [ctypes.c_void_p, ctypes.c_int, c_dblp]
lib.hyteg_lumped_mass.restype = ctypes.c_int
lib.hyteg_dirichlet_mask.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
lib.hyteg_dirichlet_mask.restype = ctypes.c_int
lib.hyteg_solver_setup.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double]
lib.hyteg_solver_setup.restype = ctypes.c_int
for _f in (lib.hyteg_restrict, lib.hyteg_prolong_add):
    _f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    _f.restype = ctypes.c_int
lib.hyteg_vcycle.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                             ctypes.c_void_p]
lib.hyteg_vcycle.restype = ctypes.c_int
lib.hyteg_solve.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                            ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_double)]
lib.hyteg_solve.restype = ctypes.c_int
lib.hyteg_last_error.argtypes = []
lib.hyteg_last_error.restype = ctypes.c_char_p
lib.hyteg_version.argtypes = []
lib.hyteg_version.restype = ctypes.c_char_p

# status codes, dtypes, boundary modes (values of include/hyteg.h)
OK, EINVAL, ENOMEM, ECUDA, EMESH, ESTATE = 0, -1, -2, -3, -4, -5
F64, F32, F64_IEEE = 1, 2, 3
BC_NONE, BC_DIRICHLET = 0, 1
SOLVE_F64, SOLVE_MIXED = 1, 2


class HytegError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = lib.hyteg_last_error().decode(errors="replace")
        super().__init__(f"{where} failed with code {code}: {msg}")


def check(code: int, where: str) -> None:
    if code != OK:
        raise HytegError(code, where)
