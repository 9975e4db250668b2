"""CPU oracle for the matrix-free P1 operator apply — TEST INFRASTRUCTURE ONLY.

Only the tests, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg
import this package.  The product path (the C-ABI library and its Python
binding) never calls it; it shares no code with the CUDA path.

What it computes, and from which passage of Thönnes & Rüde, "Model-Based
Performance Analysis of the HyTeG Finite Element Framework" (PASC '23):

* `refine`   — uniform refinement of every macro-triangle / macro-tet of an
  unstructured coarse mesh to level L (Sec. 1.2), the global numbering of the
  refined vertices and the per-macro triangular array layout (Sec. 4, the
  generated vertex-to-vertex kernel; DoF counts of Sec. 3.1).
* `assemble` — the P1 stiffness matrix of the refined mesh assembled from
  element matrices into compressed row storage (Sec. 1.1, Sec. 3), Dirichlet
  rows, and y = A x.  The paper's stencil apply reaches exactly this product:
  the constant stencil of a macro IS the matrix row of its interior points
  (Sec. 1.2, Sec. 3).
* `layout`   — the paper's closed-form DoF counts and memory volumes (Sec. 3.1,
  Table "memory level 10") and the triangular index map.
* `p2`       — the P2 (vertex + edge DoF) stiffness of the refined 2D mesh:
  the discretisation whose vertex-to-vertex, edge-to-vertex, vertex-to-edge
  and edge-to-edge kernels the paper analyses (Sec. 3.1, Sec. 5.2-5.5),
  assembled from quadratic element matrices.
* `multigrid` — a textbook V-cycle on the refinement hierarchy (levels as the
  multigrid hierarchy, Sec. 1.2; smoothers, Sec. 5.1): linear prolongation,
  R = P^T, weighted Jacobi, direct coarsest solve, lumped-mass right-hand
  side.

Everything is float64 and deliberately plain: per-element matrices, a sparse
sum of duplicates, a row loop product.  Parity pins live in tests/ (run with
`-m "not gpu"`).
"""
from .layout import (
    vertex_dofs_per_macro,
    edge_dofs_per_orientation,
    p2_dofs_per_macro,
    tri_index,
    tet_index,
    slots_per_macro,
)
from .refine import RefinedMesh
from .assemble import (
    element_stiffness,
    assemble_stiffness,
    apply_dirichlet_rows,
    operator_matrix,
    spmv,
    row_apply,
)

__all__ = [
    "vertex_dofs_per_macro",
    "edge_dofs_per_orientation",
    "p2_dofs_per_macro",
    "tri_index",
    "tet_index",
    "slots_per_macro",
    "RefinedMesh",
    "element_stiffness",
    "assemble_stiffness",
    "apply_dirichlet_rows",
    "operator_matrix",
    "spmv",
    "row_apply",
]
