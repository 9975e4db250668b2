"""Python view of a refined mesh and its operator apply (marshalling only)."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _capi as C
from ._capi import F64, F32, F64_IEEE, BC_NONE, BC_DIRICHLET, SOLVE_F64, SOLVE_MIXED, HytegError

_ELEM = {F64: 8, F32: 4, F64_IEEE: 8}


def version() -> str:
    return C.lib.hyteg_version().decode()


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Mesh:
    """A coarse simplex mesh (2D triangles / 3D tetrahedra) refined uniformly.

    coords: float64 [n_verts, dim]; cells: int64 [n_cells, dim+1] (vertex
    order inside a cell fixes the macro's local axes); bc: BC_DIRICHLET
    (identity rows on the domain boundary) or BC_NONE.
    """

    def __init__(self, coords, cells, bc: int = BC_DIRICHLET):
        coords = np.ascontiguousarray(coords, dtype=np.float64)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        if coords.ndim != 2 or cells.ndim != 2:
            raise ValueError("coords and cells must be 2-D arrays")
        self.dim = int(coords.shape[1])
        self.n_cells = int(cells.shape[0])
        h = ctypes.c_void_p()
        C.check(C.lib.hyteg_mesh_create(self.dim, coords.shape[0], coords.ctypes.data_as(C.c_dblp),
                                        cells.shape[0], cells.ctypes.data_as(C.c_i64p), bc, ctypes.byref(h)),
                "hyteg_mesh_create")
        self._h = h
        self.max_level = -1

    def close(self) -> None:
        if getattr(self, "_h", None):
            C.lib.hyteg_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def refine(self, max_level: int) -> "Mesh":
        C.check(C.lib.hyteg_mesh_refine(self._h, max_level), "hyteg_mesh_refine")
        self.max_level = max(self.max_level, max_level)
        return self

    def autotune_choice(self, level: int, dtype: int = F64) -> int:
        """z-ranges per macro-tet the 3D slab autotuner picked (0: not tuned)."""
        v = ctypes.c_int()
        C.check(C.lib.hyteg_autotune_choice(self._h, level, dtype, ctypes.byref(v)), "hyteg_autotune_choice")
        return v.value

    def num_slots(self, level: int):
        """(slots in the library layout, distinct refined vertices)."""
        ns, ng = ctypes.c_int64(), ctypes.c_int64()
        C.check(C.lib.hyteg_num_slots(self._h, level, ctypes.byref(ns), ctypes.byref(ng)), "hyteg_num_slots")
        return ns.value, ng.value

    def dof_map(self, level: int) -> np.ndarray:
        """Global vertex id of every slot (int64 [n_slots])."""
        ns, _ = self.num_slots(level)
        out = np.empty(ns, dtype=np.int64)
        C.check(C.lib.hyteg_dof_map(self._h, level, out.ctypes.data_as(C.c_i64p)), "hyteg_dof_map")
        return out

    @staticmethod
    def _dtype_code(t, ieee: bool) -> int:
        import torch
        if t.dtype == torch.float32:
            return F32
        if t.dtype == torch.float64:
            return F64_IEEE if ieee else F64
        raise TypeError(f"unsupported dtype {t.dtype}")

    def apply(self, level: int, x, y, ieee: bool = False, stream=None):
        """y = A x for device tensors x, y (float64 or float32) in slot layout.

        Enqueued on `stream` (default: torch's current stream); returns y."""
        if not (x.is_cuda and y.is_cuda):
            raise ValueError("x and y must be CUDA tensors; use apply_host for host buffers")
        if x.dtype != y.dtype or not x.is_contiguous() or not y.is_contiguous():
            raise ValueError("x and y must be contiguous and of the same dtype")
        ns, _ = self.num_slots(level)
        if x.numel() != ns or y.numel() != ns:
            raise ValueError(f"x and y must have {ns} elements")
        code = self._dtype_code(x, ieee)
        C.check(C.lib.hyteg_apply(self._h, level, code, ctypes.c_void_p(x.data_ptr()),
                                  ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))),
                "hyteg_apply")
        return y

    def apply_raw(self, level: int, dtype: int, x_ptr: int, y_ptr: int, stream_ptr: int) -> None:
        """y = A x for raw device pointers (no checks beyond the library's)."""
        C.check(C.lib.hyteg_apply(self._h, level, dtype, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr),
                                  ctypes.c_void_p(stream_ptr)), "hyteg_apply")

    def apply_timed(self, level: int, dtype: int, x_ptr: int, y_ptr: int, stream_ptr: int,
                    ev_begin: int, ev_mid: int, ev_end: int) -> None:
        """apply_raw that also records three CUDA events (raw cudaEvent_t
        handles) around the macro-interior and the interface kernel."""
        C.check(C.lib.hyteg_apply_timed(self._h, level, dtype, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr),
                                        ctypes.c_void_p(stream_ptr), ctypes.c_void_p(ev_begin),
                                        ctypes.c_void_p(ev_mid), ctypes.c_void_p(ev_end)), "hyteg_apply_timed")

    def apply_host(self, level: int, x_host, y_host, ieee: bool = False, stream=None):
        """y_host = A x_host for host tensors (pinned for full copy speed);
        copies, applies and synchronises inside the library."""
        if x_host.is_cuda or y_host.is_cuda:
            raise ValueError("apply_host takes host tensors")
        ns, _ = self.num_slots(level)
        if x_host.numel() != ns or y_host.numel() != ns or x_host.dtype != y_host.dtype:
            raise ValueError(f"x_host and y_host must have {ns} elements of one dtype")
        code = self._dtype_code(x_host, ieee)
        C.check(C.lib.hyteg_apply_host(self._h, level, code, ctypes.c_void_p(x_host.data_ptr()),
                                       ctypes.c_void_p(y_host.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))),
                "hyteg_apply_host")
        return y_host

    # ---- geometry -------------------------------------------------------------
    def apply_host_batch(self, level: int, xs_host, ys_host, ieee: bool = False, stream=None):
        """ys_host[i] = A xs_host[i] for lists of host tensors (page-locked for
        overlap), copies and applies pipelined inside the library."""
        if len(xs_host) != len(ys_host):
            raise ValueError("xs_host and ys_host differ in length")
        code = self._dtype_code(xs_host[0], ieee) if xs_host else F64
        n = len(xs_host)
        xp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in xs_host])
        yp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in ys_host])
        C.check(C.lib.hyteg_apply_host_batch(self._h, level, code, xp, yp, n, ctypes.c_void_p(_stream_ptr(stream))),
                "hyteg_apply_host_batch")
        return ys_host

    def slot_coords(self, level: int) -> np.ndarray:
        """Coordinates of every slot, float64 [n_slots, dim]."""
        ns, _ = self.num_slots(level)
        out = np.empty((ns, self.dim), dtype=np.float64)
        C.check(C.lib.hyteg_slot_coords(self._h, level, out.ctypes.data_as(C.c_dblp)), "hyteg_slot_coords")
        return out

    def lumped_mass(self, level: int) -> np.ndarray:
        """Lumped P1 mass of every slot (copies hold the full value)."""
        ns, _ = self.num_slots(level)
        out = np.empty(ns, dtype=np.float64)
        C.check(C.lib.hyteg_lumped_mass(self._h, level, out.ctypes.data_as(C.c_dblp)), "hyteg_lumped_mass")
        return out

    def dirichlet_mask(self, level: int) -> np.ndarray:
        """True for every slot of a Dirichlet DoF."""
        ns, _ = self.num_slots(level)
        out = np.empty(ns, dtype=np.uint8)
        C.check(C.lib.hyteg_dirichlet_mask(self._h, level, ctypes.c_void_p(out.ctypes.data)), "hyteg_dirichlet_mask")
        return out.astype(bool)

    # ---- multigrid --------------------------------------------------------------
    def solver_setup(self, max_level: int, nu1: int = 3, nu2: int = 3, omega: float = 2.0 / 3.0) -> "Mesh":
        C.check(C.lib.hyteg_solver_setup(self._h, max_level, nu1, nu2, omega), "hyteg_solver_setup")
        return self

    def restrict(self, fine_level: int, r_fine, b_coarse, stream=None):
        code = self._dtype_code(r_fine, False)
        C.check(C.lib.hyteg_restrict(self._h, fine_level, code, ctypes.c_void_p(r_fine.data_ptr()),
                                     ctypes.c_void_p(b_coarse.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))),
                "hyteg_restrict")
        return b_coarse

    def prolong_add(self, fine_level: int, e_coarse, u_fine, stream=None):
        code = self._dtype_code(u_fine, False)
        C.check(C.lib.hyteg_prolong_add(self._h, fine_level, code, ctypes.c_void_p(e_coarse.data_ptr()),
                                        ctypes.c_void_p(u_fine.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))),
                "hyteg_prolong_add")
        return u_fine

    def vcycle(self, level: int, b, u, stream=None):
        code = self._dtype_code(u, False)
        C.check(C.lib.hyteg_vcycle(self._h, level, code, ctypes.c_void_p(b.data_ptr()),
                                   ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))),
                "hyteg_vcycle")
        return u

    def solve(self, level: int, b, u, mode: int = SOLVE_MIXED, rtol: float = 1e-10, max_iter: int = 100,
              stream=None):
        """Solve A u = b (float64 device tensors, u = initial guess);
        returns (iterations, relative residual)."""
        it, rel = ctypes.c_int(), ctypes.c_double()
        C.check(C.lib.hyteg_solve(self._h, level, mode, ctypes.c_void_p(b.data_ptr()),
                                  ctypes.c_void_p(u.data_ptr()), rtol, max_iter,
                                  ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(it), ctypes.byref(rel)),
                "hyteg_solve")
        return it.value, rel.value

    def solve_two_part(self, level: int, b, u, u_lo, mode: int = SOLVE_MIXED, rtol: float = 1e-10,
                       max_iter: int = 100, stream=None):
        """Solve A (u + u_lo) = b with an iterate of two float64 device
        tensors (u_lo: the low part, zeros to start); returns (iterations,
        relative residual of u + u_lo)."""
        it, rel = ctypes.c_int(), ctypes.c_double()
        C.check(C.lib.hyteg_solve_two_part(self._h, level, mode, ctypes.c_void_p(b.data_ptr()),
                                           ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(u_lo.data_ptr()), rtol,
                                           max_iter, ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(it),
                                           ctypes.byref(rel)),
                "hyteg_solve_two_part")
        return it.value, rel.value

    # ---- Poisson model problem -------------------------------------------------
    def poisson_rhs(self, level: int, seed: int, noise: float, b, stream=None):
        """b (float64 device tensor, slot layout) = lumped mass * (prod sin(pi p)
        + noise * Philox normal of the global DoF id), 0 on Dirichlet DoFs."""
        C.check(C.lib.hyteg_poisson_rhs(self._h, level, seed, noise, ctypes.c_void_p(b.data_ptr()),
                                        ctypes.c_void_p(_stream_ptr(stream))), "hyteg_poisson_rhs")
        return b

    def to_global(self, level: int, v, v_global, stream=None):
        """v_global[gid] = v (float64 device tensors)."""
        C.check(C.lib.hyteg_to_global(self._h, level, ctypes.c_void_p(v.data_ptr()),
                                      ctypes.c_void_p(v_global.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))),
                "hyteg_to_global")
        return v_global

    # ---- P2 (vertex + edge DoFs, 2D) ---------------------------------------------
    def p2_num_slots(self, level: int):
        ns, ng = ctypes.c_int64(), ctypes.c_int64()
        C.check(C.lib.hyteg_p2_num_slots(self._h, level, ctypes.byref(ns), ctypes.byref(ng)), "hyteg_p2_num_slots")
        return ns.value, ng.value

    def p2_dof_map(self, level: int) -> np.ndarray:
        ns, _ = self.p2_num_slots(level)
        out = np.empty(ns, dtype=np.int64)
        C.check(C.lib.hyteg_p2_dof_map(self._h, level, out.ctypes.data_as(C.c_i64p)), "hyteg_p2_dof_map")
        return out

    def p2_apply(self, level: int, x, y, ieee: bool = False, stream=None):
        """y = A x with the P2 stiffness (device tensors of P2 slots)."""
        code = self._dtype_code(x, ieee)
        C.check(C.lib.hyteg_p2_apply(self._h, level, code, ctypes.c_void_p(x.data_ptr()),
                                     ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))),
                "hyteg_p2_apply")
        return y

    def p2_apply_timed(self, level: int, dtype: int, x_ptr: int, y_ptr: int, stream_ptr: int,
                       ev_begin: int, ev_mid: int, ev_end: int) -> None:
        """P2 apply on raw pointers recording three raw cudaEvent_t handles
        around the merged apply kernel and the interface kernels."""
        C.check(C.lib.hyteg_p2_apply_timed(self._h, level, dtype, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr),
                                           ctypes.c_void_p(stream_ptr), ctypes.c_void_p(ev_begin),
                                           ctypes.c_void_p(ev_mid), ctypes.c_void_p(ev_end)), "hyteg_p2_apply_timed")


def apply_batch(meshes, levels, xs, ys, ieee: bool = False, stream=None):
    """ys[i] = A_i xs[i] for several (mesh, level) products in as few launches
    as possible: the 2D ones share one kernel launch per 64 meshes.  All
    vectors are contiguous CUDA tensors of one dtype; returns ys."""
    n = len(meshes)
    if not (len(levels) == len(xs) == len(ys) == n):
        raise ValueError("meshes, levels, xs and ys must have the same length")
    if n == 0:
        return ys
    dt = xs[0].dtype
    for M, lev, x, y in zip(meshes, levels, xs, ys):
        if not (x.is_cuda and y.is_cuda) or x.dtype != dt or y.dtype != dt:
            raise ValueError("all vectors must be CUDA tensors of one dtype")
        if not (x.is_contiguous() and y.is_contiguous()):
            raise ValueError("vectors must be contiguous")
        ns, _ = M.num_slots(lev)
        if x.numel() != ns or y.numel() != ns:
            raise ValueError(f"vectors of level {lev} must have {ns} elements")
    code = Mesh._dtype_code(xs[0], ieee)
    hs = (ctypes.c_void_p * n)(*[M._h.value if isinstance(M._h, ctypes.c_void_p) else M._h for M in meshes])
    ls = (ctypes.c_int * n)(*levels)
    xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    yp = (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys])
    C.check(C.lib.hyteg_apply_batch(hs, ls, code, xp, yp, n, ctypes.c_void_p(_stream_ptr(stream))),
            "hyteg_apply_batch")
    return ys



def solve_two_part_group(meshes, level: int, bs, us, u_los, mode: int = SOLVE_MIXED, rtol: float = 1e-10,
                         max_iter: int = 100, stream=None):
    """Solve A_i (u_i + u_lo_i) = b_i for several meshes at one level in
    lockstep (hyteg_solve_two_part_group): every solve step is one launch for
    all problems still iterating.  bs, us, u_los: float64 CUDA tensors in the
    slot layout of each mesh.  Returns [(iterations, relative residual)]."""
    n = len(meshes)
    if not (len(bs) == len(us) == len(u_los) == n):
        raise ValueError("meshes, bs, us and u_los must have the same length")
    if n == 0:
        return []
    for M, b, u, lo in zip(meshes, bs, us, u_los):
        ns, _ = M.num_slots(level)
        for v in (b, u, lo):
            if not v.is_cuda or v.dtype.itemsize != 8 or not v.is_contiguous() or v.numel() != ns:
                raise ValueError(f"vectors must be contiguous float64 CUDA tensors of {ns} elements")
    hs = (ctypes.c_void_p * n)(*[M._h.value if isinstance(M._h, ctypes.c_void_p) else M._h for M in meshes])
    bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in bs])
    up = (ctypes.c_void_p * n)(*[u.data_ptr() for u in us])
    lp = (ctypes.c_void_p * n)(*[u.data_ptr() for u in u_los])
    it = (ctypes.c_int * n)()
    rel = (ctypes.c_double * n)()
    C.check(C.lib.hyteg_solve_two_part_group(hs, n, level, mode, bp, up, lp, rtol, max_iter,
                                             ctypes.c_void_p(_stream_ptr(stream)), it, rel),
            "hyteg_solve_two_part_group")
    return [(it[i], rel[i]) for i in range(n)]
