"""The synthetic request stream of the solve-server workload.

Requests arrive as a Poisson process (exponential inter-arrival times of mean
1/rate); half are 2D and half 3D.  A 2D request solves on a rectangle of
kx x ky square cells of two triangles each, (kx, ky) uniform over the pairs with
2 <= kx*ky <= 32 (4..64 macro-triangles), at a level uniform in 5..10; a 3D
request on a box of kx x ky x kz cubic cells of six Kuhn tetrahedra,
(kx, ky, kz) uniform over the triples with kx*ky*kz <= 64 (6..384
macro-tets), at a level uniform in 3..6.  Coarse meshes are jittered (0.15 of
the cell width in 2D, 0.1 in 3D) with mesh seed 0, so requests of one shape
share their coarse mesh; every request has its own right-hand-side seed.
Everything is drawn from PCG64(seed) in request order.
"""
from __future__ import annotations

from dataclasses import dataclass
from functools import lru_cache

import numpy as np

from .meshes import rect_mesh, box_kuhn_mesh, CoarseMesh


@dataclass(frozen=True)
class Request:
    index: int
    arrival_s: float
    dim: int
    shape: tuple
    level: int
    rhs_seed: int


def _pairs():
    return [(a, b) for a in range(1, 33) for b in range(1, 33) if 2 <= a * b <= 32]


def _triples():
    return [(a, b, c) for a in range(1, 65) for b in range(1, 65) for c in range(1, 65) if a * b * c <= 64]


def request_stream(n: int, rate: float = 2000.0, seed: int = 3) -> list[Request]:
    rng = np.random.Generator(np.random.PCG64(seed))
    pairs, triples = _pairs(), _triples()
    out, t = [], 0.0
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        if rng.random() < 0.5:
            shape = pairs[rng.integers(len(pairs))]
            out.append(Request(i, t, 2, shape, int(rng.integers(5, 11)), 1000 + i))
        else:
            shape = triples[rng.integers(len(triples))]
            out.append(Request(i, t, 3, shape, int(rng.integers(3, 7)), 1000 + i))
    return out


@lru_cache(maxsize=None)
def coarse_mesh(dim: int, shape: tuple) -> CoarseMesh:
    if dim == 2:
        return rect_mesh(shape[0], shape[1], 0.15, 0, square_cells=True)
    return box_kuhn_mesh(shape[0], shape[1], shape[2], 0.1, 0, cube_cells=True)
