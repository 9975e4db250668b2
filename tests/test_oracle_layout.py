"""Oracle layout and counts pinned to numbers the paper prints (CPU only)."""
import os

import numpy as np
import pytest

import oracle
from oracle.refine import local_points
from inputs import unit_square_mesh, unit_cube_kuhn_mesh

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


def test_dof_counts_table_level10():
    g = {k: int(v) for k, v in _read("dof_counts_level10.txt")}
    assert oracle.vertex_dofs_per_macro(10) == g["vertex"]
    assert oracle.edge_dofs_per_orientation(10) == g["edge_per_orientation"]
    assert oracle.p2_dofs_per_macro(10) == g["dof"]
    assert 8 * oracle.p2_dofs_per_macro(10) == g["dof_mem_bytes"]
    assert 8 * g["entries_per_vertex_stencil"] * oracle.vertex_dofs_per_macro(10) == g["vertex_stencil_mem_bytes"]
    assert 8 * g["entries_per_edge_stencil"] * 3 * oracle.edge_dofs_per_orientation(10) == g["edge_stencil_mem_bytes"]
    # the P1 array of one macro holds exactly the vertex DoFs
    assert oracle.slots_per_macro(2, 10) == g["vertex"]


def test_generated_kernel_index_expressions_level10():
    rows = [[int(v) for v in r] for r in _read("vtv_index_level10.txt")]
    assert sorted(r[0] for r in rows) == list(range(7))
    T = lambda m: m * (m + 1) // 2
    rng = np.random.default_rng(0)
    ys = rng.integers(1, 1023, size=400)
    xs = np.array([rng.integers(1, 1024 - y) for y in ys])
    for slot, q, c, dx, dy in rows:
        paper = xs + 1026 * ys - T(ys + q) + c
        ours = oracle.tri_index(xs + dx, ys + dy, 10)
        np.testing.assert_array_equal(ours, paper, err_msg=f"slot {slot}")
    # destination index
    np.testing.assert_array_equal(oracle.tri_index(xs, ys, 10), xs + 1026 * ys - T(ys))


def test_generated_kernel_loop_bounds_are_the_macro_interior():
    # 1 <= y < 2^L, 1 <= x < 2^L - y  visits exactly the points strictly inside
    for L in range(2, 8):
        n = 1 << L
        pts = {(x, y) for y in range(1, n) for x in range(1, n - y)}
        rm = oracle.RefinedMesh(*_sq(1), L)
        assert len(pts) == rm.n_cell_pts == (n - 1) * (n - 2) // 2


def _sq(k, jit=0.0):
    m = unit_square_mesh(k, jit, 0)
    return m.coords, m.cells


def _cube(k, jit=0.0):
    m = unit_cube_kuhn_mesh(k, jit, 0)
    return m.coords, m.cells


@pytest.mark.parametrize("L", [0, 1, 2, 3])
def test_array_order_is_row_major_x_inner(L):
    n = 1 << L
    pts2 = local_points(2, n)
    np.testing.assert_array_equal(oracle.tri_index(pts2[:, 0], pts2[:, 1], L), np.arange(len(pts2)))
    pts3 = local_points(3, n)
    np.testing.assert_array_equal(oracle.tet_index(pts3[:, 0], pts3[:, 1], pts3[:, 2], L), np.arange(len(pts3)))
    # brute-force order: z outer, y, x inner
    brute = [(x, y, z) for z in range(n + 1) for y in range(n + 1 - z) for x in range(n + 1 - z - y)]
    np.testing.assert_array_equal(pts3, np.array(brute).reshape(-1, 3))


@pytest.mark.parametrize("k,L", [(1, 0), (1, 3), (2, 2), (4, 3)])
def test_unique_dofs_of_unit_square(k, L):
    rm = oracle.RefinedMesh(*_sq(k, 0.15), L)
    assert rm.n_global == (k * (1 << L) + 1) ** 2
    smap = rm.slot_map()
    assert np.array_equal(np.unique(smap), np.arange(rm.n_global))


@pytest.mark.parametrize("k,L", [(1, 0), (1, 2), (2, 2)])
def test_unique_dofs_of_unit_cube(k, L):
    rm = oracle.RefinedMesh(*_cube(k, 0.1), L)
    assert rm.n_global == (k * (1 << L) + 1) ** 3
    smap = rm.slot_map()
    assert np.array_equal(np.unique(smap), np.arange(rm.n_global))


@pytest.mark.parametrize("dim,k,L", [(2, 4, 3), (3, 2, 2)])
def test_macro_copies_share_position(dim, k, L):
    """Every slot's position through its macro's affine map equals the
    position of the global point it is numbered as."""
    rm = oracle.RefinedMesh(*(_sq(k, 0.15) if dim == 2 else _cube(k, 0.1)), L)
    for m in range(rm.cells.shape[0]):
        v = rm.coarse_coords[rm.cells[m]]
        pos = v[0] + (rm.local / rm.n) @ (v[1:] - v[0])
        g = rm.local_to_global(m, rm.local)
        np.testing.assert_allclose(pos, rm.coords[g], atol=1e-14)


def test_boundary_flags_unit_square():
    rm = oracle.RefinedMesh(*_sq(4, 0.15), 3)
    on_edge = np.any((np.abs(rm.coords) < 1e-14) | (np.abs(rm.coords - 1) < 1e-14), axis=1)
    np.testing.assert_array_equal(rm.boundary, on_edge)


def test_boundary_flags_unit_cube():
    rm = oracle.RefinedMesh(*_cube(2, 0.1), 2)
    on_face = np.any((np.abs(rm.coords) < 1e-14) | (np.abs(rm.coords - 1) < 1e-14), axis=1)
    np.testing.assert_array_equal(rm.boundary, on_face)


def test_kuhn_refinement_counts():
    for L in range(0, 4):
        rm = oracle.RefinedMesh(*_cube(1), L)
        ntets = sum(v.shape[0] for m in range(6) for v in rm.elements(m))
        assert ntets == 6 * 8 ** L
        rm2 = oracle.RefinedMesh(*_sq(1), L)
        ntri = sum(v.shape[0] for m in range(2) for v in rm2.elements(m))
        assert ntri == 2 * 4 ** L
