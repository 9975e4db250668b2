"""P1 stiffness assembly, Dirichlet rows and y = A x (oracle side).

Test infrastructure only; see the package docstring.

The paper compares its matrix-free stencil apply with an assembled sparse
matrix in compressed row storage (Sec. 1.1 "Sparse Matrices", Sec. 3): both
give the same product, since the stencil of a macro is the matrix row of each
of its interior points (Sec. 1.2, Sec. 3).  This module builds that matrix the
textbook way:

* element matrix of a simplex T with vertices P_0..P_d:
  K_T = |T| G^T G, where column i of G is the gradient of the barycentric
  coordinate lambda_i; with J = [P_1-P_0, ..., P_d-P_0] the gradients of
  lambda_1..lambda_d are the columns of J^{-T} and grad lambda_0 = -sum of the
  others; |T| = |det J| / d!;
* global matrix = sum of element matrices (COO duplicates summed into CSR);
* Dirichlet: the rows of domain-boundary DoFs become identity rows (y_b = x_b);
  interior rows keep their boundary columns.

Element edge vectors are formed from the macro's affine map and the integer
index differences of the element's vertices (P(q) - P(q') = M (q - q') / n),
which keeps them accurate to one rounding even at level 11, where micro
edges are ~1e-4 long.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from .refine import RefinedMesh, element_offsets, in_region


def element_stiffness(J: np.ndarray) -> np.ndarray:
    """P1 Laplace element matrices for a stack of edge matrices J [k, d, d]
    (column i = P_{i+1} - P_0).  Returns [k, d+1, d+1]."""
    J = np.asarray(J, dtype=np.float64)
    if J.ndim == 2:
        J = J[None]
    k, d, _ = J.shape
    det = np.linalg.det(J)
    vol = np.abs(det) / math.factorial(d)
    JinvT = np.transpose(np.linalg.inv(J), (0, 2, 1))  # columns: grad lambda_1..d
    G = np.empty((k, d, d + 1))
    G[:, :, 1:] = JinvT
    G[:, :, 0] = -JinvT.sum(axis=2)
    return vol[:, None, None] * np.einsum("kai,kaj->kij", G, G)


def _macro_element_matrices(rm: RefinedMesh, m: int, verts: np.ndarray) -> np.ndarray:
    """Element matrices of the micro-elements of macro m whose local vertex
    index points are verts [k, d+1, d]."""
    M = rm.macro_matrix(m)  # d x d, columns v_i - v_0
    D = (verts[:, 1:, :] - verts[:, :1, :]).astype(np.float64)  # [k, d(edges), d(index)]
    # edge vector j = M @ D[j] / n ; J columns are edge vectors
    J = np.einsum("ab,kjb->kaj", M, D) / rm.n
    return element_stiffness(J)


def assemble_stiffness(rm: RefinedMesh) -> sp.csr_matrix:
    """Global P1 stiffness matrix without boundary conditions (CSR, float64)."""
    rows, cols, vals = [], [], []
    d = rm.dim
    for m in range(rm.cells.shape[0]):
        for verts in rm.elements(m):
            if verts.shape[0] == 0:
                continue
            K = _macro_element_matrices(rm, m, verts)
            g = rm.local_to_global(m, verts.reshape(-1, d)).reshape(-1, d + 1)
            rows.append(np.repeat(g, d + 1, axis=1).ravel())
            cols.append(np.tile(g, (1, d + 1)).ravel())
            vals.append(K.ravel())
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    A = sp.coo_matrix((vals, (rows, cols)), shape=(rm.n_global, rm.n_global)).tocsr()
    A.sum_duplicates()
    return A


def apply_dirichlet_rows(A: sp.csr_matrix, boundary: np.ndarray) -> sp.csr_matrix:
    """Replace the rows of boundary DoFs by identity rows."""
    keep = sp.diags((~boundary).astype(np.float64))
    ident = sp.diags(boundary.astype(np.float64))
    return (keep @ A + ident).tocsr()


def operator_matrix(rm: RefinedMesh) -> sp.csr_matrix:
    """The operator the apply computes: stiffness with Dirichlet identity rows."""
    return apply_dirichlet_rows(assemble_stiffness(rm), rm.boundary)


def spmv(A: sp.csr_matrix, x: np.ndarray) -> np.ndarray:
    """y = A x in float64 (compressed-row product: one pass over the rows)."""
    return A @ np.asarray(x, dtype=np.float64)


# ---------------------------------------------------------------------------
# Row-by-row evaluation for sampled checks at sizes too large to assemble.
# ---------------------------------------------------------------------------

def _incidences(rm: RefinedMesh, gid: int):
    """(macro, local point) pairs of every macro copy of global point gid."""
    d, n = rm.dim, rm.n
    E = np.vstack([np.zeros(d, dtype=np.int64), np.eye(d, dtype=np.int64)])  # corner index vectors
    out = []
    cells = rm.cells
    if gid < rm.base_edge:
        v = gid
        for m in np.nonzero((cells == v).any(axis=1))[0]:
            i = int(np.nonzero(cells[m] == v)[0][0])
            out.append((int(m), n * E[i]))
    elif gid < rm.base_face:
        e, r = divmod(gid - rm.base_edge, rm.n_edge_pts)
        k = r + 1
        lo, hi = rm.edges[e]
        for m in np.nonzero((cells == lo).any(axis=1) & (cells == hi).any(axis=1))[0]:
            ilo = int(np.nonzero(cells[m] == lo)[0][0])
            ihi = int(np.nonzero(cells[m] == hi)[0][0])
            out.append((int(m), (n - k) * E[ilo] + k * E[ihi]))
    elif gid < rm.base_cell:
        f, r = divmod(gid - rm.base_face, rm.n_face_pts)
        # decode (a, b): rows b = 1.., row b holds n-1-b points
        b = 1
        while r >= n - 1 - b:
            r -= n - 1 - b
            b += 1
        a = r + 1
        f0, f1, f2 = rm.faces[f]
        inc = (cells == f0).any(axis=1) & (cells == f1).any(axis=1) & (cells == f2).any(axis=1)
        for m in np.nonzero(inc)[0]:
            i0, i1, i2 = (int(np.nonzero(cells[m] == v)[0][0]) for v in (f0, f1, f2))
            out.append((int(m), (n - a - b) * E[i0] + a * E[i1] + b * E[i2]))
    else:
        m, r = divmod(gid - rm.base_cell, rm.n_cell_pts)
        pos = int(np.nonzero(rm._interior_rank == r)[0][0])
        out.append((int(m), rm.local[pos]))
    return out


def row_apply(rm: RefinedMesh, gids, x: np.ndarray) -> np.ndarray:
    """(A x)[g] for each global id g, with A = operator_matrix(rm), computed
    one row at a time from the micro-elements that contain the point."""
    offsets = element_offsets(rm.dim)
    d = rm.dim
    res = np.empty(len(gids), dtype=np.float64)
    for t, g in enumerate(gids):
        g = int(g)
        if rm.boundary[g]:
            res[t] = x[g]
            continue
        acc = 0.0
        for m, p in _incidences(rm, g):
            for off in offsets:
                for r in range(d + 1):
                    verts = (p - off[r])[None, :] + off  # element with p as vertex r
                    if not np.all(in_region(verts, rm.n)):
                        continue
                    K = _macro_element_matrices(rm, m, verts[None])[0]
                    gv = rm.local_to_global(m, verts)
                    acc += float(K[r] @ x[gv])
        res[t] = acc
    return res
