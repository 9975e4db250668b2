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
lib.hyteg_autotune_choice.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
lib.hyteg_autotune_choice.restype = ctypes.c_int
lib.hyteg_apply_batch.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                  ctypes.c_void_p]
lib.hyteg_apply_batch.restype = ctypes.c_int
lib.hyteg_num_slots.argtypes = [ctypes.c_void_p, ctypes.c_int, c_i64p, c_i64p]
lib.hyteg_num_slots.restype = ctypes.c_int
lib.hyteg_dof_map.argtypes = [ctypes.c_void_p, ctypes.c_int, c_i64p]
lib.hyteg_dof_map.restype = ctypes.c_int
lib.hyteg_apply.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                            ctypes.c_void_p]
lib.hyteg_apply.restype = ctypes.c_int
lib.hyteg_apply_partial.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p]
lib.hyteg_apply_partial.restype = ctypes.c_int
lib.hyteg_apply_timed.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
lib.hyteg_apply_timed.restype = ctypes.c_int
lib.hyteg_apply_host.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p]
lib.hyteg_apply_host.restype = ctypes.c_int
lib.hyteg_apply_host_batch.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                       ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p]
lib.hyteg_apply_host_batch.restype = ctypes.c_int
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
lib.hyteg_solve_two_part.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
lib.hyteg_solve_two_part.restype = ctypes.c_int
lib.hyteg_solve_two_part_group.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                           ctypes.POINTER(ctypes.c_void_p), ctypes.c_double, ctypes.c_int,
                                           ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_double)]
lib.hyteg_solve_two_part_group.restype = ctypes.c_int
lib.hyteg_p2_num_slots.argtypes = [ctypes.c_void_p, ctypes.c_int, c_i64p, c_i64p]
lib.hyteg_p2_num_slots.restype = ctypes.c_int
lib.hyteg_p2_dof_map.argtypes = [ctypes.c_void_p, ctypes.c_int, c_i64p]
lib.hyteg_p2_dof_map.restype = ctypes.c_int
lib.hyteg_p2_apply.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_void_p]
lib.hyteg_p2_apply.restype = ctypes.c_int
lib.hyteg_p2_apply_timed.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]
lib.hyteg_p2_apply_timed.restype = ctypes.c_int
lib.hyteg_poisson_rhs.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p,
                                  ctypes.c_void_p]
lib.hyteg_poisson_rhs.restype = ctypes.c_int
lib.hyteg_to_global.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
lib.hyteg_to_global.restype = ctypes.c_int


class Request(ctypes.Structure):
    """struct hyteg_request"""
    _fields_ = [("dim", ctypes.c_int), ("n_verts", ctypes.c_int64), ("coords", c_dblp), ("n_cells", ctypes.c_int64),
                ("cells", c_i64p), ("level", ctypes.c_int), ("mode", ctypes.c_int), ("rtol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("seed", ctypes.c_uint64), ("noise", ctypes.c_double),
                ("u_out", c_dblp), ("b_out", c_dblp), ("u_lo_out", c_dblp)]


class Result(ctypes.Structure):
    """struct hyteg_result"""
    _fields_ = [("status", ctypes.c_int), ("error", ctypes.c_int), ("iters", ctypes.c_int),
                ("cache_hit", ctypes.c_int), ("relres", ctypes.c_double), ("queue_s", ctypes.c_double),
                ("run_s", ctypes.c_double), ("n_global", ctypes.c_int64), ("setup_s", ctypes.c_double),
                ("group", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    """struct hyteg_server_stats"""
    _fields_ = [("submitted", ctypes.c_int64), ("done", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("in_flight", ctypes.c_int64), ("cached_meshes", ctypes.c_int64), ("cache_hits", ctypes.c_int64),
                ("evictions", ctypes.c_int64), ("reserved_bytes", ctypes.c_size_t), ("arena_used", ctypes.c_size_t),
                ("group_solves", ctypes.c_int64), ("grouped", ctypes.c_int64)]


lib.hyteg_server_create.argtypes = [ctypes.c_int, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
lib.hyteg_server_create.restype = ctypes.c_int
lib.hyteg_server_submit.argtypes = [ctypes.c_void_p, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
lib.hyteg_server_submit.restype = ctypes.c_int
lib.hyteg_server_poll.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(Result)]
lib.hyteg_server_poll.restype = ctypes.c_int
lib.hyteg_server_wait.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(Result)]
lib.hyteg_server_wait.restype = ctypes.c_int
lib.hyteg_server_release.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
lib.hyteg_server_release.restype = ctypes.c_int
lib.hyteg_server_stats_get.argtypes = [ctypes.c_void_p, ctypes.POINTER(ServerStats)]
lib.hyteg_server_stats_get.restype = ctypes.c_int
lib.hyteg_server_inject_alloc_failures.argtypes = [ctypes.c_void_p, ctypes.c_int]
lib.hyteg_server_inject_alloc_failures.restype = ctypes.c_int
lib.hyteg_server_destroy.argtypes = [ctypes.c_void_p]
lib.hyteg_server_destroy.restype = None
lib.hyteg_last_error.argtypes = []
lib.hyteg_last_error.restype = ctypes.c_char_p
lib.hyteg_version.argtypes = []
lib.hyteg_version.restype = ctypes.c_char_p

# status codes, dtypes, boundary modes (values of include/hyteg.h)
OK, EINVAL, ENOMEM, ECUDA, EMESH, ESTATE, EAGAIN, ETIMEDOUT = 0, -1, -2, -3, -4, -5, -6, -7
REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3
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
