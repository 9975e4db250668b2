"""Uniform refinement of a coarse simplex mesh and the global vertex numbering.

Test infrastructure only; see the package docstring.

Sec. 1.2 of the paper: every macro-triangle (macro-tet in 3D) of an
unstructured coarse mesh is refined uniformly L times, which yields a
structured grid inside each macro.  With n = 2^L intervals per macro edge, the
refined vertex with local index point q (integer, q_i >= 0, sum q_i <= n) of a
macro with vertices v_0..v_d sits at v_0 + sum_i (q_i / n)(v_i - v_0).

Micro-elements of a macro:
* 2D: "up" triangles (x,y),(x+1,y),(x,y+1) and "down" triangles
  (x+1,y),(x,y+1),(x+1,y+1) — the regular refinement drawn in Sec. 1.2.
* 3D (the paper names 3D as future work, Sec. 7): Kuhn/Freudenthal simplices
  of the index map u = (x+y+z, y+z, z); each unit u-cube splits into the six
  simplices a, a+e_p, a+e_p+e_q, a+(1,1,1), kept when inside the macro.  This
  is Bey's regular refinement with n^3 tets per macro.

Global numbering (one fixed convention; the library implements the same one
independently):
1. coarse vertices, in input order;
2. interior points of every coarse edge; edges sorted by (low id, high id);
   point k = 1..n-1 sits at v_low + (k/n)(v_high - v_low);
3. (3D) interior points of every coarse face; faces sorted by their sorted
   vertex triple (f0<f1<f2); point (a, b), a,b >= 1, a+b <= n-1, sits at
   f0 + (a/n)(f1-f0) + (b/n)(f2-f0), b outer, a inner;
4. interior points of every cell in cell order, in the cell's own array order
   (y outer / x inner in 2D; z, y, x in 3D).

Dirichlet boundary: a coarse edge (2D) or face (3D) with exactly one incident
cell is on the domain boundary; every refined vertex on it is a boundary DoF.
"""
from __future__ import annotations

from itertools import combinations, permutations

import numpy as np

from .layout import slots_per_macro, tri_index, tet_index


def local_points(dim: int, n: int) -> np.ndarray:
    """All local index points of one macro in array order, int64 [S, dim]."""
    pts = []
    if dim == 2:
        for y in range(n + 1):
            x = np.arange(n + 1 - y)
            pts.append(np.stack([x, np.full_like(x, y)], axis=1))
    else:
        for z in range(n + 1):
            for y in range(n + 1 - z):
                x = np.arange(n + 1 - z - y)
                pts.append(np.stack([x, np.full_like(x, y), np.full_like(x, z)], axis=1))
    return np.concatenate(pts, axis=0).astype(np.int64)


def element_offsets(dim: int):
    """Vertex offsets (in local index space, relative to an anchor point) of
    every micro-element type of a refined macro.  Returns a list of int64
    arrays of shape [dim+1, dim]."""
    if dim == 2:
        up = np.array([[0, 0], [1, 0], [0, 1]], dtype=np.int64)
        down = np.array([[1, 0], [0, 1], [1, 1]], dtype=np.int64)
        return [up, down]
    types = []
    for perm in permutations(range(3)):
        u = [np.zeros(3, dtype=np.int64)]
        cur = np.zeros(3, dtype=np.int64)
        for ax in perm:
            cur = cur.copy()
            cur[ax] += 1
            u.append(cur)
        u = np.array(u)
        # u -> x index: x = u1 - u2, y = u2 - u3, z = u3
        xs = np.stack([u[:, 0] - u[:, 1], u[:, 1] - u[:, 2], u[:, 2]], axis=1)
        types.append(xs)
    return types


def in_region(pts: np.ndarray, n: int) -> np.ndarray:
    """True where local index points lie in the closed macro (q >= 0, sum <= n)."""
    return np.all(pts >= 0, axis=-1) & (pts.sum(axis=-1) <= n)


class RefinedMesh:
    """The coarse mesh refined to `level`, with global numbering and geometry.

    Attributes (n = 2^level):
      dim, level, n, coarse_coords [V,dim], cells [C,dim+1]
      edges [E,2] (sorted pairs), faces [F,3] (3D, sorted triples)
      n_global, coords [n_global, dim], boundary [n_global] bool
    """

    def __init__(self, coarse_coords, cells, level: int, dirichlet: bool = True):
        self.coarse_coords = np.asarray(coarse_coords, dtype=np.float64)
        self.cells = np.asarray(cells, dtype=np.int64)
        self.dim = self.coarse_coords.shape[1]
        d = self.dim
        assert self.cells.shape[1] == d + 1
        self.level = level
        self.n = n = 1 << level
        V = self.coarse_coords.shape[0]
        C = self.cells.shape[0]

        # --- coarse topology -------------------------------------------------
        edge_set = set()
        face_set = set()
        for c in self.cells:
            for a, b in combinations(sorted(c.tolist()), 2):
                edge_set.add((a, b))
            if d == 3:
                for t in combinations(sorted(c.tolist()), 3):
                    face_set.add(t)
        self.edges = np.array(sorted(edge_set), dtype=np.int64).reshape(-1, 2)
        self.edge_index = {tuple(e): i for i, e in enumerate(self.edges.tolist())}
        self.faces = np.array(sorted(face_set), dtype=np.int64).reshape(-1, 3)
        self.face_index = {tuple(f): i for i, f in enumerate(self.faces.tolist())}

        # incidence counts for the boundary test
        top = self.edges if d == 2 else self.faces
        top_index = self.edge_index if d == 2 else self.face_index
        count = np.zeros(len(top), dtype=np.int64)
        for c in self.cells:
            for t in combinations(sorted(c.tolist()), d):
                count[top_index[t]] += 1
        bnd_top = (count == 1) if dirichlet else np.zeros(len(top), dtype=bool)
        self.bnd_vertex = np.zeros(V, dtype=bool)
        self.bnd_edge = np.zeros(len(self.edges), dtype=bool)
        self.bnd_face = np.zeros(len(self.faces), dtype=bool)
        for i in np.nonzero(bnd_top)[0]:
            verts = top[i].tolist()
            self.bnd_vertex[verts] = True
            for a, b in combinations(sorted(verts), 2):
                self.bnd_edge[self.edge_index[(a, b)]] = True
            if d == 3:
                self.bnd_face[i] = True

        # --- global numbering offsets -------------------------------------------
        self.n_edge_pts = max(n - 1, 0)
        self.n_face_pts = max((n - 1) * (n - 2) // 2, 0)
        if d == 2:
            self.n_cell_pts = self.n_face_pts
        else:
            self.n_cell_pts = max((n - 1) * (n - 2) * (n - 3) // 6, 0)
        self.base_edge = V
        self.base_face = V + len(self.edges) * self.n_edge_pts
        nf = len(self.faces) * self.n_face_pts if d == 3 else 0
        self.base_cell = self.base_face + nf
        self.n_global = self.base_cell + C * self.n_cell_pts

        self.local = local_points(d, n)
        assert self.local.shape[0] == slots_per_macro(d, level)
        interior = np.all(self.local >= 1, axis=1) & (self.local.sum(axis=1) <= n - 1)
        self._interior_rank = np.full(self.local.shape[0], -1, dtype=np.int64)
        self._interior_rank[interior] = np.arange(int(interior.sum()))

        # --- geometry and boundary flags of every global point ------------------
        self.coords = np.zeros((self.n_global, d), dtype=np.float64)
        self.boundary = np.zeros(self.n_global, dtype=bool)
        cc = self.coarse_coords
        self.coords[:V] = cc
        self.boundary[:V] = self.bnd_vertex
        if n > 1:
            k = np.arange(1, n, dtype=np.float64)
            for e, (lo, hi) in enumerate(self.edges.tolist()):
                g0 = self.base_edge + e * self.n_edge_pts
                self.coords[g0:g0 + n - 1] = cc[lo] + (k[:, None] / n) * (cc[hi] - cc[lo])
                self.boundary[g0:g0 + n - 1] = self.bnd_edge[e]
        if d == 3 and self.n_face_pts > 0:
            ab = np.array([(a, b) for b in range(1, n - 1) for a in range(1, n - b)],
                          dtype=np.float64)
            for f, (f0, f1, f2) in enumerate(self.faces.tolist()):
                g0 = self.base_face + f * self.n_face_pts
                self.coords[g0:g0 + self.n_face_pts] = (
                    cc[f0] + (ab[:, :1] / n) * (cc[f1] - cc[f0]) + (ab[:, 1:] / n) * (cc[f2] - cc[f0]))
                self.boundary[g0:g0 + self.n_face_pts] = self.bnd_face[f]
        if self.n_cell_pts > 0:
            q = self.local[interior].astype(np.float64)
            for m in range(C):
                v = cc[self.cells[m]]
                g0 = self.base_cell + m * self.n_cell_pts
                self.coords[g0:g0 + self.n_cell_pts] = v[0] + (q / n) @ (v[1:] - v[0])

    # ------------------------------------------------------------------------
    def macro_matrix(self, m: int) -> np.ndarray:
        """Columns v_i - v_0 of macro m's affine map (dim x dim)."""
        v = self.coarse_coords[self.cells[m]]
        return (v[1:] - v[0]).T

    def local_to_global(self, m: int, pts: np.ndarray) -> np.ndarray:
        """Global ids of local index points `pts` [k, dim] of macro m."""
        d, n = self.dim, self.n
        pts = np.asarray(pts, dtype=np.int64).reshape(-1, d)
        W = np.concatenate([(n - pts.sum(axis=1))[:, None], pts], axis=1)  # weight per corner
        assert np.all(W >= 0), "point outside macro"
        corners = self.cells[m]
        nz = W > 0
        code = (nz * (1 << np.arange(d + 1))).sum(axis=1)
        out = np.full(pts.shape[0], -1, dtype=np.int64)
        for c in np.unique(code):
            sel = code == c
            idx = [i for i in range(d + 1) if (c >> i) & 1]
            if len(idx) == 1:
                out[sel] = corners[idx[0]]
            elif len(idx) == 2:
                i, j = idx
                a, b = int(corners[i]), int(corners[j])
                lo, hi = min(a, b), max(a, b)
                e = self.edge_index[(lo, hi)]
                col_hi = i if a == hi else j
                k = W[sel, col_hi]
                out[sel] = self.base_edge + e * self.n_edge_pts + k - 1
            elif len(idx) == 3 and d == 3:
                g = sorted((int(corners[i]), i) for i in idx)
                f = self.face_index[(g[0][0], g[1][0], g[2][0])]
                a = W[sel, g[1][1]]
                b = W[sel, g[2][1]]
                within = (b - 1) * (n - 1) - ((b - 1) * b) // 2 + (a - 1)
                out[sel] = self.base_face + f * self.n_face_pts + within
            else:  # interior of the cell itself
                out[sel] = self.base_cell + m * self.n_cell_pts + self._interior_rank_of(pts[sel])
        return out

    def _interior_rank_of(self, pts: np.ndarray) -> np.ndarray:
        """Rank of interior local points among the macro's interior points in
        array order: look up the point's array position, then its rank."""
        if self.dim == 2:
            pos = tri_index(pts[:, 0], pts[:, 1], self.level)
        else:
            pos = tet_index(pts[:, 0], pts[:, 1], pts[:, 2], self.level)
        r = self._interior_rank[pos]
        assert np.all(r >= 0)
        return r

    def slot_map(self) -> np.ndarray:
        """Global id of every array slot of every macro, macros concatenated
        in cell order (the library's layout): int64 [C * S]."""
        return np.concatenate([self.local_to_global(m, self.local)
                               for m in range(self.cells.shape[0])])

    def elements(self, m: int):
        """Micro-elements of macro m: list of (local vertex points [k, d+1, d])
        per element type."""
        out = []
        for off in element_offsets(self.dim):
            verts = self.local[:, None, :] + off[None, :, :]
            keep = np.all(in_region(verts, self.n), axis=1)
            out.append(verts[keep])
        return out
