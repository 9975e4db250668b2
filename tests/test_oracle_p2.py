"""Pins of the P2 (vertex + edge DoF) oracle against what the paper and the
mathematics fix.  No GPU.  A planted mistake in the element matrix (on the
CPU) must fail at least one pin."""
import numpy as np
import pytest
import sympy

import oracle.p2 as p2
from inputs import rect_mesh, unit_square_mesh
from oracle.layout import vertex_dofs_per_macro, edge_dofs_per_orientation


# ---------------------------------------------------------------- pins
def pin_reference_element():
    """The element matrix of the reference triangle equals the exact
    integrals of the P2 basis gradients, done symbolically."""
    x, y = sympy.symbols("x y")
    lam = [1 - x - y, x, y]
    basis = [lam[i] * (2 * lam[i] - 1) for i in range(3)] + [4 * lam[0] * lam[1], 4 * lam[1] * lam[2],
                                                           4 * lam[0] * lam[2]]
    grads = [(sympy.diff(f, x), sympy.diff(f, y)) for f in basis]
    K = np.zeros((6, 6))
    for a in range(6):
        for b in range(6):
            g = grads[a][0] * grads[b][0] + grads[a][1] * grads[b][1]
            K[a, b] = float(sympy.integrate(sympy.integrate(g, (y, 0, 1 - x)), (x, 0, 1)))
    got = p2.p2_element_stiffness(np.eye(2))[0]
    np.testing.assert_allclose(got, K, rtol=0, atol=1e-14)


def _quadratic(c):
    return lambda P: c[0] + c[1] * P[:, 0] + c[2] * P[:, 1] + c[3] * P[:, 0] ** 2 + c[4] * P[:, 0] * P[:, 1] \
        + c[5] * P[:, 1] ** 2


def pin_quadratic_energy():
    """P2 interpolates quadratics exactly, so u^T K u = integral of |grad u|^2
    over the unit square for every quadratic u (jittered interior vertices)."""
    c = [1.0, 2.0, -3.0, 0.7, -1.1, 0.4]
    X, Y = sympy.symbols("X Y")
    q = c[0] + c[1] * X + c[2] * Y + c[3] * X ** 2 + c[4] * X * Y + c[5] * Y ** 2
    exact = float(sympy.integrate(sympy.diff(q, X) ** 2 + sympy.diff(q, Y) ** 2, (X, 0, 1), (Y, 0, 1)))
    for coarse, L in ((rect_mesh(3, 2, 0.15, 4), 2), (unit_square_mesh(2, 0.15, 1), 3)):
        pm = p2.P2Mesh(coarse.coords, coarse.cells, L, dirichlet=False)
        u = _quadratic(c)(pm.coords())
        K = pm.stiffness()
        assert abs(u @ (K @ u) - exact) <= 1e-11 * exact


def pin_pde_consistency():
    """For u = x^2 + y^2 (Laplace u = 4): (K u)_i = -4 * integral of phi_i at
    interior DoFs: 0 for vertex DoFs (a P2 vertex function integrates to 0 on
    every triangle), -4 * (sum of incident |T|)/3 for edge DoFs; linear u
    gives 0 at every interior DoF."""
    coarse = rect_mesh(3, 2, 0.15, 4)
    pm = p2.P2Mesh(coarse.coords, coarse.cells, 3, dirichlet=True)
    K = pm.stiffness()
    P = pm.coords()
    inner = ~pm.boundary
    r = K @ (P[:, 0] ** 2 + P[:, 1] ** 2)
    area = np.abs(np.linalg.det(pm.tri_J)) / 2.0
    edge_int = np.zeros(pm.n_global)
    np.add.at(edge_int, pm.tri_edges.ravel(), np.repeat(area / 3.0, 3))
    want = -4.0 * edge_int
    np.testing.assert_allclose(r[inner], want[inner], rtol=0, atol=1e-12)
    r_lin = K @ (0.3 + 1.7 * P[:, 0] - 0.9 * P[:, 1])
    np.testing.assert_allclose(r_lin[inner], 0.0, atol=1e-12)


def pin_row_structure():
    """Symmetric, zero row sums, 19 entries in an interior vertex row (7
    vertices + 12 edges) and 9 in an interior edge row (4 vertices + 4 edges
    + itself) (Sec. 3.1)."""
    coarse = unit_square_mesh(2, 0.15, 0)
    pm = p2.P2Mesh(coarse.coords, coarse.cells, 3, dirichlet=True)
    K = pm.stiffness()
    assert abs(K - K.T).max() < 1e-14
    np.testing.assert_allclose(np.asarray(K.sum(axis=1)).ravel(), 0.0, atol=1e-12)
    nnz = np.diff(K.indptr)
    inner = ~pm.boundary
    assert set(nnz[:pm.n_vertex][inner[:pm.n_vertex]]) == {19}
    assert set(nnz[pm.n_vertex:][inner[pm.n_vertex:]]) == {9}


def pin_counts():
    """Per-macro DoF counts of the paper at level 10 (Table "memory level
    10") and the unique DoF counts of a refined mesh."""
    assert vertex_dofs_per_macro(10) == 525825
    assert edge_dofs_per_orientation(10) == 524800
    one = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    for L in (1, 2, 3):
        pm = p2.P2Mesh(one, np.array([[0, 1, 2]]), L)
        n = 1 << L
        assert pm.n_vertex == (n + 1) * (n + 2) // 2
        assert pm.n_edge == 3 * n * (n + 1) // 2
    coarse = unit_square_mesh(2)
    pm = p2.P2Mesh(coarse.coords, coarse.cells, 2)
    assert pm.n_global == (2 * 2 * 4 + 1) ** 2  # a uniform grid of spacing h/2


# Couplings printed in the paper's listings (Sec. 5.3-5.5), as (group, dx, dy)
# offsets from the lattice point (x, y) of the target DoF; [y][x] indexing.
# Reading: the X-group term of row y+1 reads x-1 instead of x in the
# edge-to-vertex listing and the vertex term of row y+1 reads x instead of x-1
# in the vertex-to-edge listing of X (the geometry of the refinement fixes
# both; every other printed term is kept as printed).
LISTING = {
    "V": {("X", -1, 1), ("X", 0, 0), ("X", -1, 0), ("X", 0, -1),
          ("Y", -1, 0), ("Y", 0, 0), ("Y", 0, -1), ("Y", 1, -1),
          ("XY", -1, 0), ("XY", 0, 0), ("XY", -1, -1), ("XY", 0, -1),
          ("V", 0, 0), ("V", 1, 0), ("V", -1, 0), ("V", 0, 1), ("V", 0, -1), ("V", 1, -1), ("V", -1, 1)},
    "X": {("V", 0, 1), ("V", 0, 0), ("V", 1, 0), ("V", 1, -1),
          ("X", 0, 0), ("Y", 0, 0), ("Y", 1, -1), ("XY", 0, 0), ("XY", 0, -1)},
    "XY": {("V", 0, 1), ("V", 1, 1), ("V", 0, 0), ("V", 1, 0),
           ("XY", 0, 0), ("X", 0, 0), ("X", 0, 1), ("Y", 0, 0), ("Y", 1, 0)},
    "Y": {("V", -1, 1), ("V", 0, 1), ("V", 0, 0), ("V", 1, 0),
          ("Y", 0, 0), ("X", 0, 0), ("X", -1, 1), ("XY", 0, 0), ("XY", -1, 0)},
}


def pin_listing_couplings():
    """Inside a macro every DoF couples exactly with the DoFs of the paper's
    four kernel listings (vertex-to-vertex shape of Sec. 5.2; edge-to-vertex,
    vertex-to-edge and edge-to-edge of Sec. 5.3-5.5)."""
    one = np.array([[0.0, 0.0], [1.0, 0.1], [0.3, 0.9]])
    L, n = 3, 8
    pm = p2.P2Mesh(one, np.array([[0, 1, 2]]), L, dirichlet=False)
    smap = pm.slot_map()
    K = pm.stiffness()
    nv = vertex_dofs_per_macro(L)
    ne = edge_dofs_per_orientation(L)

    def slot(group, x, y):
        if group == "V":
            return x + y * (n + 1) - (y * (y - 1)) // 2
        base = nv + {"X": 0, "Y": 1, "XY": 2}[group] * ne
        return base + y * n - (y * (y - 1)) // 2 + x

    x0, y0 = 3, 2
    for tgt, want in LISTING.items():
        row = K.getrow(smap[slot(tgt, x0, y0)])
        # structural couplings: for the Laplacian the vertex-to-opposite-edge
        # entries of an element matrix are exactly zero, but they are couplings
        # of the element (the listings carry them as weights)
        got = set(row.indices.tolist())
        expect = {int(smap[slot(g, x0 + dx, y0 + dy)]) for g, dx, dy in want}
        assert got == expect, tgt


def pin_opposite_couplings_vanish():
    """For the Laplacian a vertex does not couple with the edge opposite to it
    in a triangle: the integral of (4 lambda_i - 1) lambda_k over T is
    4|T|/12 - |T|/3 = 0.  In the assembled matrix the vertex row has six and
    every edge row two rounding-sized entries, at the opposite couplings."""
    coarse = rect_mesh(3, 2, 0.15, 4)
    pm = p2.P2Mesh(coarse.coords, coarse.cells, 3, dirichlet=False)
    K = pm.stiffness().tocoo()
    scale = np.abs(K.data).max()
    # (vertex, edge) pairs that share a triangle with the edge opposite the vertex
    opp = set()
    for tv, te in zip(pm.tri_vertices.tolist(), pm.tri_edges.tolist()):
        for v, e in zip(tv, (te[1], te[2], te[0])):  # e12 opposite v0, e02 opposite v1, e01 opposite v2
            opp.add((v, e))
    inc = set()
    for tv, te in zip(pm.tri_vertices.tolist(), pm.tri_edges.tolist()):
        for v in tv:
            for e, ends in zip(te, ((tv[0], tv[1]), (tv[1], tv[2]), (tv[0], tv[2]))):
                if v in ends:
                    inc.add((v, e))
    only_opp = opp - inc
    assert only_opp
    vals = {(int(r), int(c)): v for r, c, v in zip(K.row, K.col, K.data)}
    for v, e in only_opp:
        assert abs(vals[(v, e)]) <= 1e-14 * scale
        assert abs(vals[(e, v)]) <= 1e-14 * scale


ALL_PINS = [("reference_element", pin_reference_element), ("quadratic_energy", pin_quadratic_energy),
            ("pde_consistency", pin_pde_consistency), ("row_structure", pin_row_structure),
            ("counts", pin_counts), ("listing_couplings", pin_listing_couplings),
            ("opposite_couplings_vanish", pin_opposite_couplings_vanish)]


@pytest.mark.parametrize("name,check", ALL_PINS, ids=[n for n, _ in ALL_PINS])
def test_pin(name, check):
    check()


def test_dirichlet_rows_and_slot_map():
    coarse = rect_mesh(2, 1, 0.15, 3)
    pm = p2.P2Mesh(coarse.coords, coarse.cells, 2)
    A = pm.operator_matrix()
    b = np.nonzero(pm.boundary)[0]
    for g in b[:20]:
        row = A.getrow(g)
        assert row.nnz == 1 and row.indices[0] == g and row.data[0] == 1.0
    smap = pm.slot_map()
    assert set(smap.tolist()) == set(range(pm.n_global))
    # boundary edges have one copy, interface edges two, the rest one
    cnt = np.bincount(smap, minlength=pm.n_global)
    assert cnt.max() <= 6 and cnt[pm.n_vertex:].max() == 2


# ------------------------------------------------------- planted mistakes
def _mutant(vertex=(4.0, -1.0), edge=4.0, weight=1.0 / 3.0):
    def f(J):
        J = np.asarray(J, dtype=np.float64)
        if J.ndim == 2:
            J = J[None]
        area = np.abs(np.linalg.det(J)) / 2.0
        JinvT = np.transpose(np.linalg.inv(J), (0, 2, 1))
        g = np.empty((J.shape[0], 2, 3))
        g[:, :, 1:] = JinvT
        g[:, :, 0] = -JinvT.sum(axis=2)
        K = np.zeros((J.shape[0], 6, 6))
        for lam in ([0.5, 0.5, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5]):
            grads = np.empty((J.shape[0], 6, 2))
            for a, (i, j) in enumerate(p2._NODES):
                if i == j:
                    grads[:, a, :] = (vertex[0] * lam[i] + vertex[1]) * g[:, :, i]
                else:
                    grads[:, a, :] = edge * (lam[j] * g[:, :, i] + lam[i] * g[:, :, j])
            K += (area * weight)[:, None, None] * np.einsum("kad,kbd->kab", grads, grads)
        return K
    f.__name__ = f"mutant_v{vertex}_e{edge}_w{weight:.3f}"
    return f


MUTANTS = [_mutant(vertex=(4.0, 1.0)), _mutant(vertex=(2.0, -1.0)), _mutant(edge=2.0), _mutant(weight=0.5)]


def test_unmutated_builder_matches():
    J = np.array([[[0.3, -0.1], [0.2, 0.5]]])
    np.testing.assert_allclose(_mutant()(J), p2.p2_element_stiffness(J), rtol=0, atol=1e-15)


@pytest.mark.parametrize("mutant", MUTANTS, ids=lambda f: f.__name__)
def test_planted_mistakes_fail_a_pin(mutant, monkeypatch):
    monkeypatch.setattr(p2, "p2_element_stiffness", mutant)
    failed = []
    for name, check in ALL_PINS:
        try:
            check()
        except AssertionError:
            failed.append(name)
    assert failed, f"{mutant.__name__} passed every pin"
