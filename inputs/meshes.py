"""Coarse meshes and random vectors for the synthetic workloads.

The coarse meshes follow the workloads the method is measured on: the unit
square split into right triangles (two macro-triangles for the smallest case,
4x4 cells x 2 triangles with jittered interior vertices for the large 2D case)
and the unit cube split into Kuhn tetrahedra (4x4x4 cells x 6 tets with
jittered interior vertices).  The paper refines such macro-triangles uniformly
to level L (Sec. 1.2, "Hybrid Tetrahedral Grids"); the refinement itself is NOT
done here.

Vertex order inside each cell is part of the input: 2D triangles list the
right-angle vertex first and are counter-clockwise; 3D tets follow the monotone
Kuhn path corner -> +e_a -> +e_a+e_b -> opposite corner.
"""
from __future__ import annotations

from dataclasses import dataclass
from itertools import permutations

import numpy as np


@dataclass(frozen=True)
class CoarseMesh:
    """An unstructured coarse mesh of simplices.

    coords: float64 [n_verts, dim]; cells: int64 [n_cells, dim+1].
    """

    dim: int
    coords: np.ndarray
    cells: np.ndarray
    name: str = ""

    @property
    def n_verts(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_cells(self) -> int:
        return int(self.cells.shape[0])


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _jitter_interior(coords: np.ndarray, amplitude: float, seed: int, hi=1.0) -> np.ndarray:
    """Move every vertex not on the boundary of the box [0, hi] by U[-a, a] per
    coordinate, drawn in ascending vertex-id order (x, y[, z] per vertex)."""
    if amplitude == 0.0:
        return coords
    on_bnd = np.any((coords <= 0.0) | (coords >= np.asarray(hi)), axis=1)
    interior = np.nonzero(~on_bnd)[0]
    d = _rng(seed).uniform(-amplitude, amplitude, size=(interior.size, coords.shape[1]))
    out = coords.copy()
    out[interior] += d
    return out


def unit_square_mesh(k: int, jitter: float = 0.0, seed: int = 0) -> CoarseMesh:
    """k x k cells of the unit square, each split along its (0,0)-(1,1)
    diagonal into two right triangles (see `rect_mesh`)."""
    return rect_mesh(k, k, jitter, seed)


def rect_mesh(kx: int, ky: int, jitter: float = 0.0, seed: int = 0, square_cells: bool = False) -> CoarseMesh:
    """kx x ky cells, each split along its (0,0)-(1,1) diagonal into two
    triangles: cells of the unit square, or (square_cells) square cells of
    side 1/max(kx, ky) filling the rectangle [0, kx/k] x [0, ky/k].

    Vertex id of grid point (i, j) is i + (kx+1) j.  For cell (i, j) with
    corners a=(i,j), b=(i+1,j), c=(i,j+1), d=(i+1,j+1) the triangles are
    (b, d, a) and (c, a, d): right angle (for square cells) first,
    counter-clockwise.  Cells are listed cell-row by cell-row, lower-right
    triangle first.  `jitter` is the amplitude as a fraction of the smaller
    cell width 1/max(kx, ky).
    """
    k = max(kx, ky)
    hx, hy = (kx / k, ky / k) if square_cells else (1.0, 1.0)
    gx = np.linspace(0.0, hx, kx + 1)
    gy = np.linspace(0.0, hy, ky + 1)
    xx, yy = np.meshgrid(gx, gy, indexing="xy")
    coords = np.stack([xx.ravel(), yy.ravel()], axis=1).astype(np.float64)
    cells = []
    for j in range(ky):
        for i in range(kx):
            a = i + (kx + 1) * j
            b = a + 1
            c = a + (kx + 1)
            d = c + 1
            cells.append((b, d, a))
            cells.append((c, a, d))
    coords = _jitter_interior(coords, jitter / k, seed, (hx, hy))
    name = (f"square{kx}x{ky}" if kx == ky else f"rect{kx}x{ky}" + ("sq" if square_cells else "")) + (f"_jit{jitter}_s{seed}" if jitter else "")
    return CoarseMesh(2, coords, np.asarray(cells, dtype=np.int64), name)


def unit_cube_kuhn_mesh(k: int, jitter: float = 0.0, seed: int = 0) -> CoarseMesh:
    """k x k x k cells of the unit cube, each split into the 6 Kuhn tetrahedra
    that share the cell's main diagonal (see `box_kuhn_mesh`)."""
    return box_kuhn_mesh(k, k, k, jitter, seed)


def box_kuhn_mesh(kx: int, ky: int, kz: int, jitter: float = 0.0, seed: int = 0,
                  cube_cells: bool = False) -> CoarseMesh:
    """kx x ky x kz cells, each split into the 6 Kuhn tetrahedra that share
    the cell's main diagonal: cells of the unit cube, or (cube_cells) cubes of
    side 1/max(kx, ky, kz) filling the box [0, kx/k] x [0, ky/k] x [0, kz/k].

    Vertex id of grid point (i, j, l) is i + (kx+1) j + (kx+1)(ky+1) l.  The
    tet of a permutation (p, q, r) of the axes has vertices corner,
    corner + e_p, corner + e_p + e_q, corner + (1,1,1), in that order.
    Permutations are taken in itertools order; cells are listed cell by cell
    (i fastest).  `jitter` is a fraction of the smallest cell width.
    """
    k = max(kx, ky, kz)
    hx, hy, hz = (kx / k, ky / k, kz / k) if cube_cells else (1.0, 1.0, 1.0)
    gx = np.linspace(0.0, hx, kx + 1)
    gy = np.linspace(0.0, hy, ky + 1)
    gz = np.linspace(0.0, hz, kz + 1)
    zz, yy, xx = np.meshgrid(gz, gy, gx, indexing="ij")
    coords = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1).astype(np.float64)

    def vid(i, j, l):
        return i + (kx + 1) * j + (kx + 1) * (ky + 1) * l

    cells = []
    for l in range(kz):
        for j in range(ky):
            for i in range(kx):
                base = np.array([i, j, l])
                for perm in permutations(range(3)):
                    p0 = base.copy()
                    p1 = p0.copy()
                    p1[perm[0]] += 1
                    p2 = p1.copy()
                    p2[perm[1]] += 1
                    p3 = base + 1
                    cells.append(tuple(vid(*p) for p in (p0, p1, p2, p3)))
    coords = _jitter_interior(coords, jitter / k, seed, (hx, hy, hz))
    name = (f"cube{kx}^3kuhn" if kx == ky == kz else f"box{kx}x{ky}x{kz}kuhn" + ("cc" if cube_cells else "")) + (
        f"_jit{jitter}_s{seed}" if jitter else "")
    return CoarseMesh(3, coords, np.asarray(cells, dtype=np.int64), name)


def random_vector(n: int, seed: int, low: float = -1.0, high: float = 1.0) -> np.ndarray:
    """n float64 values ~ U[low, high) from PCG64(seed), in index order."""
    return _rng(seed).uniform(low, high, size=n)


def range_vector(n: int, seed: int, pattern: str) -> np.ndarray:
    """n float64 values from PCG64(seed) spanning the float64 range, for the
    checks of an apply's arithmetic far from magnitude 1:
      "scale:<k>"  U[-1, 1) * 2^k
      "mixed"      U[-1, 1) times 1 or 1e-30, each with probability 1/2
      "huge"       U[-1, 1) with 1 % of the entries +-U[0.5, 1) * 1e300
      "sparse"     U[-1, 1) with 90 % of the entries +0.0 or -0.0
      "subnormal"  U[-1, 1) * 2^-1040 (mostly float64 subnormals)"""
    g = _rng(seed)
    u = g.uniform(-1.0, 1.0, size=n)
    if pattern.startswith("scale:"):
        return np.ldexp(u, int(pattern.split(":")[1]))
    if pattern == "mixed":
        return np.where(g.random(n) < 0.5, u, u * 1e-30)
    if pattern == "huge":
        pick = g.random(n) < 0.01
        big = np.sign(u) * g.uniform(0.5, 1.0, size=n) * 1e300
        return np.where(pick, big, u)
    if pattern == "sparse":
        zero = g.random(n) < 0.9
        return np.where(zero, np.where(u < 0, -0.0, 0.0), u)
    if pattern == "subnormal":
        return np.ldexp(u, -1040)
    raise ValueError(f"unknown pattern {pattern!r}")


def random_normal(n: int, seed: int) -> np.ndarray:
    """n float64 values ~ N(0, 1) from PCG64(seed), in index order."""
    return _rng(seed).standard_normal(n)


# The measured workloads: coarse mesh recipe, refinement level, vector seed.
WORKLOADS = {
    # two right triangles, level 7: the small case an apply is checked on exactly
    "square2_L7": dict(dim=2, k=1, jitter=0.0, mesh_seed=0, level=7, x_seed=1),
    # 32 jittered macro-triangles, level 11 (~67M DoFs): the 2D throughput case
    "square32jit_L11": dict(dim=2, k=4, jitter=0.15, mesh_seed=0, level=11, x_seed=1),
    # the same 32 macros with P2 (vertex + edge) DoFs at level 10: as many DoFs
    # per macro as P1 at level 11 (the paper's #dof of Sec. 3.1, 67.2M slots)
    "square32jit_P2_L10": dict(dim=2, k=4, jitter=0.15, mesh_seed=0, level=10, x_seed=1, op="p2"),
    # 384 jittered Kuhn macro-tets, level 6 (~17M DoFs): the 3D throughput case
    "cube384jit_L6": dict(dim=3, k=4, jitter=0.1, mesh_seed=0, level=6, x_seed=1),
    # Poisson solve: 32 jittered macro-triangles at level 10, noise seed 2
    "square32jit_L10_solve": dict(dim=2, k=4, jitter=0.15, mesh_seed=0, level=10, x_seed=2),
}


def workload(name: str, level: int | None = None):
    """Return (CoarseMesh, level, x_seed) for a named workload; `level`
    overrides the refinement level (smaller sizes for checks)."""
    w = WORKLOADS[name]
    if w["dim"] == 2:
        mesh = unit_square_mesh(w["k"], w["jitter"], w["mesh_seed"])
    else:
        mesh = unit_cube_kuhn_mesh(w["k"], w["jitter"], w["mesh_seed"])
    return mesh, (w["level"] if level is None else level), w["x_seed"]
