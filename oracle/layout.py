"""Closed-form counts and the per-macro array index (oracle side).

Test infrastructure only; see the package docstring.
"""
from __future__ import annotations


def vertex_dofs_per_macro(level: int) -> int:
    """Vertex DoFs of one macro-triangle refined `level` times:
    (2^l + 1)(2^l + 2) / 2 (Sec. 3.1, "#vertex")."""
    n = 1 << level
    return (n + 1) * (n + 2) // 2


def edge_dofs_per_orientation(level: int) -> int:
    """Edge DoFs of ONE orientation (X, Y or XY) of a refined macro-triangle:
    2^l (2^l + 1) / 2 (Sec. 3.1, "#edge")."""
    n = 1 << level
    return n * (n + 1) // 2


def p2_dofs_per_macro(level: int) -> int:
    """#dof = #vertex + 3 #edge (Sec. 3.1)."""
    return vertex_dofs_per_macro(level) + 3 * edge_dofs_per_orientation(level)


def slots_per_macro(dim: int, level: int) -> int:
    """Array slots of one macro: every refined vertex of the closed macro,
    including its boundary copies.  2D: (n+1)(n+2)/2; 3D: (n+1)(n+2)(n+3)/6."""
    n = 1 << level
    if dim == 2:
        return (n + 1) * (n + 2) // 2
    return (n + 1) * (n + 2) * (n + 3) // 6


def tri_index(x, y, level: int):
    """Row-major index of local point (x, y) in a macro-triangle array with x
    the inner, contiguous coordinate.  Row y holds the N - y points
    x = 0..N-1-y (N = 2^l + 1 points per macro edge), so row y starts after
    sum_{k<y} (N - k) entries (Sec. 4, the array accesses of the generated
    kernel; Sec. 5, iteration starts at the right angle with x inner)."""
    N = (1 << level) + 1
    return x + y * N - (y * (y - 1)) // 2


def tet_slice_offsets(level: int):
    """Start index of every z-slice of a macro-tet array (length N+1; the last
    entry is the total slot count).  Slice z is a triangle of side N - z."""
    import numpy as np
    N = (1 << level) + 1
    sizes = [(N - k) * (N - k + 1) // 2 for k in range(N)]
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def tet_index(x, y, z, level: int):
    """Index of local point (x, y, z) in a macro-tet array: z-slices outer,
    each slice a triangular array of side N - z laid out as `tri_index`
    (x inner, then y)."""
    import numpy as np
    N = (1 << level) + 1
    off = tet_slice_offsets(level)
    z = np.asarray(z)
    Ns = N - z
    return off[z] + x + y * Ns - (y * (y - 1)) // 2
