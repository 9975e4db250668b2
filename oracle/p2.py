"""P2 (quadratic Lagrange) stiffness on the refined 2D mesh — oracle side.

Test infrastructure only; see the package docstring.

The paper's kernels belong to a discretisation with DoFs on the vertices AND
on the edges of the refined triangles (Sec. 3.1: #vertex + 3 #edge DoFs per
macro, the edges grouped into the three orientations X, Y and XY; Sec. 5.2 to
5.5: the vertex-to-vertex, edge-to-vertex, vertex-to-edge and edge-to-edge
couplings).  That is the P2 element: quadratic on every micro-triangle, one
DoF per vertex and one per edge midpoint.  This module is its plain
definition:

* element basis on a triangle with barycentric coordinates lambda_i:
  vertex i: lambda_i (2 lambda_i - 1); edge (i, j): 4 lambda_i lambda_j;
  gradients (4 lambda_i - 1) g_i and 4 (lambda_j g_i + lambda_i g_j), g_i the
  (constant) gradient of lambda_i;
* element matrix K_ab = integral over T of grad phi_a . grad phi_b, integrated
  with the three-point edge-midpoint rule (weights |T|/3), which is exact for
  the quadratic integrand;
* global matrix = sum of element matrices; the rows of DoFs on the domain
  boundary (vertices as in RefinedMesh, edges with a single incident
  micro-triangle) become identity rows.

Global numbering: the refined vertices as in RefinedMesh, then the micro-edges
sorted by their (low, high) global vertex pair.  Element DoF order:
[v0, v1, v2, e01, e12, e02].

Library layout (what the GPU path stores, used to gather into it): per macro
the vertex array (the P1 layout) followed by three edge arrays X, Y, XY of
n(n+1)/2 entries each; edge (x, y) of a group, x + y <= n-1, sits at
y n - y(y-1)/2 + x; X(x, y) joins points (x, y)-(x+1, y), Y(x, y) joins
(x, y)-(x, y+1), XY(x, y) joins (x+1, y)-(x, y+1).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .refine import RefinedMesh
from .layout import vertex_dofs_per_macro, edge_dofs_per_orientation

# local DoF -> (corner a, corner b) of the element (a == b: vertex)
_NODES = [(0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (0, 2)]


def p2_element_stiffness(J: np.ndarray) -> np.ndarray:
    """P2 Laplace element matrices for edge matrices J [k, 2, 2] (column i =
    P_{i+1} - P_0).  Returns [k, 6, 6] in the order [v0, v1, v2, e01, e12, e02]."""
    J = np.asarray(J, dtype=np.float64)
    if J.ndim == 2:
        J = J[None]
    area = np.abs(np.linalg.det(J)) / 2.0
    JinvT = np.transpose(np.linalg.inv(J), (0, 2, 1))
    g = np.empty((J.shape[0], 2, 3))
    g[:, :, 1:] = JinvT
    g[:, :, 0] = -JinvT.sum(axis=2)
    K = np.zeros((J.shape[0], 6, 6))
    # quadrature points: the edge midpoints, barycentric coordinates
    for lam in ([0.5, 0.5, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5]):
        grads = np.empty((J.shape[0], 6, 2))
        for a, (i, j) in enumerate(_NODES):
            if i == j:
                grads[:, a, :] = (4.0 * lam[i] - 1.0) * g[:, :, i]
            else:
                grads[:, a, :] = 4.0 * (lam[j] * g[:, :, i] + lam[i] * g[:, :, j])
        K += (area / 3.0)[:, None, None] * np.einsum("kad,kbd->kab", grads, grads)
    return K


class P2Mesh:
    """P2 DoFs of a 2D coarse mesh refined to `level`.

    Attributes: rm (the vertex RefinedMesh), n_vertex, edges [E, 2] (sorted
    global vertex pairs), n_edge, n_global, boundary [n_global] bool,
    tri_vertices [T, 3] and tri_edges [T, 3] (global DoF ids per micro-
    triangle, edges in the order e01, e12, e02), tri_J [T, 2, 2].
    """

    def __init__(self, coarse_coords, cells, level: int, dirichlet: bool = True):
        self.rm = rm = RefinedMesh(coarse_coords, cells, level, dirichlet=dirichlet)
        assert rm.dim == 2, "P2 is built for 2D meshes"
        self.level, self.n = level, rm.n
        tv, tj = [], []
        for m in range(rm.cells.shape[0]):
            M = rm.macro_matrix(m)
            for verts in rm.elements(m):
                if verts.shape[0] == 0:
                    continue
                tv.append(rm.local_to_global(m, verts.reshape(-1, 2)).reshape(-1, 3))
                D = (verts[:, 1:, :] - verts[:, :1, :]).astype(np.float64)
                tj.append(np.einsum("ab,kjb->kaj", M, D) / rm.n)
        self.tri_vertices = np.concatenate(tv)
        self.tri_J = np.concatenate(tj)
        pairs = np.stack([self.tri_vertices[:, [0, 1]], self.tri_vertices[:, [1, 2]],
                          self.tri_vertices[:, [0, 2]]], axis=1)  # [T, 3, 2]
        pairs = np.sort(pairs, axis=2)
        self.edges, inv, count = np.unique(pairs.reshape(-1, 2), axis=0, return_inverse=True, return_counts=True)
        self.n_vertex = rm.n_global
        self.n_edge = len(self.edges)
        self.n_global = self.n_vertex + self.n_edge
        self.tri_edges = self.n_vertex + inv.reshape(-1, 3)
        self.boundary = np.zeros(self.n_global, dtype=bool)
        self.boundary[:self.n_vertex] = rm.boundary
        if dirichlet:
            self.boundary[self.n_vertex:] = count == 1
        self._edge_id = {(int(a), int(b)): self.n_vertex + i for i, (a, b) in enumerate(self.edges.tolist())}

    def coords(self) -> np.ndarray:
        """Coordinates of every DoF: vertices, then edge midpoints."""
        c = self.rm.coords
        return np.concatenate([c, 0.5 * (c[self.edges[:, 0]] + c[self.edges[:, 1]])])

    def stiffness(self) -> sp.csr_matrix:
        K = p2_element_stiffness(self.tri_J)
        dofs = np.concatenate([self.tri_vertices, self.tri_edges], axis=1)  # [T, 6]
        rows = np.repeat(dofs, 6, axis=1).ravel()
        cols = np.tile(dofs, (1, 6)).ravel()
        A = sp.coo_matrix((K.ravel(), (rows, cols)), shape=(self.n_global, self.n_global)).tocsr()
        A.sum_duplicates()
        return A

    def operator_matrix(self) -> sp.csr_matrix:
        A = self.stiffness()
        keep = sp.diags((~self.boundary).astype(np.float64))
        ident = sp.diags(self.boundary.astype(np.float64))
        return (keep @ A + ident).tocsr()

    # ---- the library's slot layout ------------------------------------------------
    def slot_map(self) -> np.ndarray:
        """Global P2 id of every slot of every macro in the library layout."""
        rm, n = self.rm, self.n
        xs, ys = [], []
        for y in range(n):
            x = np.arange(n - y)
            xs.append(x)
            ys.append(np.full_like(x, y))
        ex, ey = np.concatenate(xs), np.concatenate(ys)
        ends = {  # local end points of the edges of each group
            "X": (np.stack([ex, ey], 1), np.stack([ex + 1, ey], 1)),
            "Y": (np.stack([ex, ey], 1), np.stack([ex, ey + 1], 1)),
            "XY": (np.stack([ex + 1, ey], 1), np.stack([ex, ey + 1], 1)),
        }
        out = []
        for m in range(rm.cells.shape[0]):
            out.append(rm.local_to_global(m, rm.local))
            for grp in ("X", "Y", "XY"):
                a = rm.local_to_global(m, ends[grp][0])
                b = rm.local_to_global(m, ends[grp][1])
                lo, hi = np.minimum(a, b), np.maximum(a, b)
                out.append(np.array([self._edge_id[(int(p), int(q))] for p, q in zip(lo, hi)], dtype=np.int64))
        s = np.concatenate(out)
        per = vertex_dofs_per_macro(self.level) + 3 * edge_dofs_per_orientation(self.level)
        assert s.size == rm.cells.shape[0] * per
        return s
