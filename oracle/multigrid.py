"""Textbook geometric multigrid on the refinement hierarchy (oracle side).

Test infrastructure only; see the package docstring.

The paper names the refinement levels as the natural multigrid hierarchy
(Sec. 1.2) and multigrid smoothers among the kernels HyTeG generates
(Sec. 5.1).  It fixes no cycle; this module takes the standard one:
* A_l: the operator of level l (P1 stiffness, Dirichlet identity rows);
* P_l: linear interpolation from level l-1 to level l — a fine vertex that
  coincides with a coarse vertex copies it, a fine vertex at the midpoint of
  a coarse micro-edge takes the mean of the edge's two end points (the
  refined P1 spaces are nested);
* restriction R_l = P_l^T, after which the Dirichlet rows of the coarse
  residual are set to zero (the correction vanishes on the boundary);
* smoother: weighted Jacobi u <- u + w D^{-1} (b - A u), w = 2/3;
* V(nu1, nu2) cycle, coarsest level 0 solved directly;
* right-hand side of -Lap u = f: lumped mass, b_i = f(p_i) |supp phi_i| / (d+1),
  zero on Dirichlet DoFs.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from .assemble import operator_matrix, assemble_stiffness
from .refine import RefinedMesh

# Kuhn edge directions in the index space (3D) and the 2D triangle edges; a
# fine vertex with parity pattern q mod 2 is the midpoint of the coarse
# micro-edge with the same parity pattern.
_EDGE_DIRS = {
    2: [(1, 0), (0, 1), (1, -1)],
    3: [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, -1, 0), (1, 0, -1), (0, 1, -1), (1, -1, 1)],
}


def prolongation(fine: RefinedMesh, coarse: RefinedMesh) -> sp.csr_matrix:
    """P: coarse (level l-1) global vector -> fine (level l) global vector."""
    d = fine.dim
    dirs = {tuple(np.mod(e, 2)): np.array(e) for e in _EDGE_DIRS[d]}
    rows, cols, vals = [], [], []
    for m in range(fine.cells.shape[0]):
        q = fine.local  # fine local points
        par = np.mod(q, 2)
        even = ~par.any(axis=1)
        gf = fine.local_to_global(m, q)
        # coincident vertices
        gc = coarse.local_to_global(m, q[even] // 2)
        rows.append(gf[even]); cols.append(gc); vals.append(np.ones(gc.size))
        # edge midpoints
        for pat, e in dirs.items():
            sel = np.all(par == np.array(pat), axis=1)
            if not sel.any():
                continue
            c1 = (q[sel] - e) // 2
            c2 = (q[sel] + e) // 2
            g1 = coarse.local_to_global(m, c1)
            g2 = coarse.local_to_global(m, c2)
            rows += [gf[sel], gf[sel]]
            cols += [g1, g2]
            vals += [np.full(g1.size, 0.5), np.full(g2.size, 0.5)]
    rows = np.concatenate(rows); cols = np.concatenate(cols); vals = np.concatenate(vals)
    # a fine vertex shared by several macros is listed once per macro with the
    # same entries: keep one copy of each (row, col)
    key = rows * coarse.n_global + cols
    _, first = np.unique(key, return_index=True)
    return sp.csr_matrix((vals[first], (rows[first], cols[first])), shape=(fine.n_global, coarse.n_global))


def lumped_mass(rm: RefinedMesh) -> np.ndarray:
    """|supp phi_i| / (d+1) for every global vertex: the row sums of the P1
    mass matrix, i.e. the volume of the incident micro-elements over d+1."""
    d = rm.dim
    mass = np.zeros(rm.n_global)
    for m in range(rm.cells.shape[0]):
        M = rm.macro_matrix(m)
        for verts in rm.elements(m):
            if verts.shape[0] == 0:
                continue
            D = (verts[:, 1:, :] - verts[:, :1, :]).astype(np.float64)
            J = np.einsum("ab,kjb->kaj", M, D) / rm.n
            vol = np.abs(np.linalg.det(J)) / (2.0 if d == 2 else 6.0)
            g = rm.local_to_global(m, verts.reshape(-1, d)).reshape(-1, d + 1)
            np.add.at(mass, g.ravel(), np.repeat(vol / (d + 1), d + 1))
    return mass


def poisson_rhs(rm: RefinedMesh, f_values: np.ndarray) -> np.ndarray:
    """b = lumped mass * f at the vertices, zero on Dirichlet DoFs."""
    b = lumped_mass(rm) * f_values
    b[rm.boundary] = 0.0
    return b


class Hierarchy:
    """Operators and transfers of levels 0..L of one coarse mesh."""

    def __init__(self, coords, cells, level: int):
        self.meshes = [RefinedMesh(coords, cells, l) for l in range(level + 1)]
        self.A = [operator_matrix(rm) for rm in self.meshes]
        self.D = [A.diagonal() for A in self.A]
        self.P = [None] + [prolongation(self.meshes[l], self.meshes[l - 1]) for l in range(1, level + 1)]
        self.level = level
        self.A0 = self.A[0].toarray()

    def smooth(self, l, u, b, sweeps, omega=2.0 / 3.0):
        A, D = self.A[l], self.D[l]
        for _ in range(sweeps):
            u = u + omega * (b - A @ u) / D
        return u

    def vcycle(self, l, u, b, nu1=3, nu2=3, omega=2.0 / 3.0):
        """One V(nu1, nu2) cycle for A_l u = b starting from u."""
        if l == 0:
            return np.linalg.solve(self.A0, b)
        u = self.smooth(l, u, b, nu1, omega)
        r = b - self.A[l] @ u
        rc = self.P[l].T @ r
        rc[self.meshes[l - 1].boundary] = 0.0
        ec = self.vcycle(l - 1, np.zeros_like(rc), rc, nu1, nu2, omega)
        u = u + self.P[l] @ ec
        return self.smooth(l, u, b, nu2, omega)

    def solve(self, b, rtol=1e-10, max_cycles=100, nu1=3, nu2=3):
        """V-cycles from u = 0 until ||b - A u|| / ||b|| <= rtol (2-norm over
        all DoFs; Dirichlet rows contribute zero).  Returns (u, history)."""
        L = self.level
        u = np.zeros_like(b)
        nb = np.linalg.norm(b)
        hist = [1.0]
        for _ in range(max_cycles):
            u = self.vcycle(L, u, b, nu1, nu2)
            hist.append(np.linalg.norm(b - self.A[L] @ u) / nb)
            if hist[-1] <= rtol:
                break
        return u, hist


# ---------------------------------------------------------------------------
# Residuals beyond float64 rounding.  A float64 vector u can only approximate
# the discrete solution u* to half an ulp per entry; its residual
# b - A fl(u*) = A (u* - fl(u*)) then sets a floor on the attainable relative
# residual, which grows like h^-2 in 2D (b shrinks like h^2 while A keeps its
# scale).  These functions measure that floor exactly and reach below it with
# an iterate of two float64 parts.
# ---------------------------------------------------------------------------

def _two_product(a: np.ndarray, b: np.ndarray):
    """a * b = p + e exactly (Dekker's product with Veltkamp's split)."""
    p = a * b
    c = 134217729.0  # 2^27 + 1
    def split(v):
        t = c * v
        hi = t - (t - v)
        return hi, v - hi
    ah, al = split(a)
    bh, bl = split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def exact_residual(A: sp.csr_matrix, b: np.ndarray, parts) -> np.ndarray:
    """r = b - A (u_1 + u_2 + ...) for float64 vectors u_k, every product
    a_ij u_kj split exactly into two float64 terms and every row summed by
    math.fsum: the correctly rounded residual of the unevaluated sum."""
    A = A.tocsr()
    chunks = []
    for u in parts:
        p, e = _two_product(A.data, np.asarray(u, dtype=np.float64)[A.indices])
        chunks.append((p, e))
    r = np.empty(A.shape[0])
    ip = A.indptr
    for i in range(A.shape[0]):
        lo, hi = ip[i], ip[i + 1]
        vals = [b[i]]
        for p, e in chunks:
            vals.extend((-p[lo:hi]).tolist())
            vals.extend((-e[lo:hi]).tolist())
        r[i] = math.fsum(vals)
    return r


def relres_exact(A: sp.csr_matrix, b: np.ndarray, parts, interior: np.ndarray) -> float:
    """||b - A sum(parts)||_2 / ||b||_2 over the rows `interior` (non-Dirichlet
    DoFs), the residual rounded once per entry."""
    r = exact_residual(A, b, parts)[interior]
    return float(np.linalg.norm(r) / np.linalg.norm(b[interior]))


def float64_floor_estimate(A: sp.csr_matrix, b: np.ndarray, u: np.ndarray, interior: np.ndarray) -> float:
    """Expected relative residual of fl(u*) when the rounding errors of the
    entries are independent and uniform in half an ulp:
    sqrt(sum_j c_j ulp(u_j)^2 / 12) / ||b||, c_j the squared column norm of
    A over the rows `interior`."""
    Ai = A.tocsr()[interior]
    c = np.asarray(Ai.multiply(Ai).sum(axis=0)).ravel()
    ulp = np.spacing(np.abs(u))
    return float(np.sqrt(np.sum(c * ulp ** 2) / 12.0) / np.linalg.norm(b[interior]))


def solve_two_part(h: "Hierarchy", b: np.ndarray, cycles: int, nu1=3, nu2=3):
    """Iterative refinement with an iterate of two float64 parts: each step
    takes the exact residual of u_hi + u_lo, one V-cycle on the residual
    equation from zero, and adds the correction to u_hi with the rounding
    error of that addition carried into u_lo (TwoSum).  Returns (u_hi, u_lo)."""
    L = h.level
    A = h.A[L]
    u_hi = np.zeros_like(b)
    u_lo = np.zeros_like(b)
    for _ in range(cycles):
        r = exact_residual(A, b, (u_hi, u_lo))
        e = h.vcycle(L, np.zeros_like(r), r, nu1, nu2)
        s = u_hi + e
        bv = s - u_hi
        err = (u_hi - (s - bv)) + (e - bv)
        u_hi = s
        u_lo = u_lo + err
    # renormalise: u_hi the float64 rounding of the sum, u_lo the rest
    s = u_hi + u_lo
    u_lo = u_lo - (s - u_hi)
    return s, u_lo
