"""The C ABI on the host: the library loads, exports every declared symbol,
and its host-side logic (mesh checks, slot counts, DoF map) agrees with the
oracle bit for bit.  No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import importlib.util
    spec = importlib.util.spec_from_file_location("hyteg_build", os.path.join(ROOT, "paper_2305_15116_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    b.build()
    import paper_2305_15116_gb300 as H
    return H


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(hyteg_\w+)\s*\(", src)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "hyteg_apply" in names and "hyteg_mesh_create" in names
    so = ctypes.CDLL(os.path.join(ROOT, "paper_2305_15116_gb300", "libhyteg.so"))
    for n in names:
        assert hasattr(so, n), f"{n} not exported"


def test_version(lib):
    assert "sm_103a" in lib.version()


from inputs import unit_square_mesh, unit_cube_kuhn_mesh
import oracle


@pytest.mark.parametrize("k,jit,L", [(1, 0.0, 0), (1, 0.0, 4), (4, 0.15, 0), (4, 0.15, 1), (4, 0.15, 5), (3, 0.1, 3)])
def test_dof_map_matches_oracle_2d(lib, k, jit, L):
    m = unit_square_mesh(k, jit, 0)
    M = lib.Mesh(m.coords, m.cells)
    rm = oracle.RefinedMesh(m.coords, m.cells, L)
    ns, ng = M.num_slots(L)
    assert ng == rm.n_global == (k * 2 ** L + 1) ** 2
    assert ns == m.n_cells * oracle.slots_per_macro(2, L)
    np.testing.assert_array_equal(M.dof_map(L), rm.slot_map())


@pytest.mark.parametrize("k,L", [(1, 0), (1, 3), (2, 2), (2, 3)])
def test_dof_map_matches_oracle_3d(lib, k, L):
    m = unit_cube_kuhn_mesh(k, 0.1, 0)
    M = lib.Mesh(m.coords, m.cells)
    rm = oracle.RefinedMesh(m.coords, m.cells, L)
    ns, ng = M.num_slots(L)
    assert ng == rm.n_global == (k * 2 ** L + 1) ** 3
    np.testing.assert_array_equal(M.dof_map(L), rm.slot_map())


def test_dof_map_any_vertex_order(lib):
    """Cells with rotated / reflected vertex order (either orientation)."""
    m = unit_square_mesh(3, 0.1, 4)
    rng = np.random.default_rng(2)
    cells = np.array([c[rng.permutation(3)] for c in m.cells])
    M = lib.Mesh(m.coords, cells)
    rm = oracle.RefinedMesh(m.coords, cells, 3)
    np.testing.assert_array_equal(M.dof_map(3), rm.slot_map())
    m3 = unit_cube_kuhn_mesh(1, 0.0, 0)
    cells3 = np.array([c[rng.permutation(4)] for c in m3.cells])
    M3 = lib.Mesh(m3.coords, cells3)
    rm3 = oracle.RefinedMesh(m3.coords, cells3, 2)
    np.testing.assert_array_equal(M3.dof_map(2), rm3.slot_map())


def test_mesh_errors(lib):
    from paper_2305_15116_gb300 import HytegError
    m = unit_square_mesh(1)
    with pytest.raises(HytegError) as e:
        lib.Mesh(m.coords, np.array([[0, 1, 1]]))
    assert e.value.code == -4  # repeated vertex
    with pytest.raises(HytegError) as e:
        lib.Mesh(np.array([[0.0, 0], [1, 0], [2, 0]]), np.array([[0, 1, 2]]))
    assert e.value.code == -4  # zero area
    with pytest.raises(HytegError) as e:
        lib.Mesh(m.coords, np.array([[0, 1, 7]]))
    assert e.value.code == -4  # id out of range
    # an edge shared by three triangles
    coords = np.array([[0.0, 0], [1, 0], [0, 1], [0, -1], [1, 1]])
    with pytest.raises(HytegError) as e:
        lib.Mesh(coords, np.array([[0, 1, 2], [0, 1, 3], [0, 1, 4]]))
    assert e.value.code == -4
    M = lib.Mesh(m.coords, m.cells)
    with pytest.raises(HytegError) as e:
        M.num_slots(16)
    assert e.value.code == -1


def test_boundary_modes_count(lib):
    m = unit_square_mesh(2, 0.1, 0)
    for bc in (0, 1):
        M = lib.Mesh(m.coords, m.cells, bc)
        assert M.num_slots(2)[1] == 81


@pytest.mark.parametrize("dim,k,L", [(2, 4, 0), (2, 4, 3), (3, 2, 2), (3, 1, 3)])
def test_slot_coords_and_lumped_mass_match_oracle(lib, dim, k, L):
    import oracle.multigrid as omg
    m = unit_square_mesh(k, 0.15, 1) if dim == 2 else unit_cube_kuhn_mesh(k, 0.1, 1)
    M = lib.Mesh(m.coords, m.cells)
    rm = oracle.RefinedMesh(m.coords, m.cells, L)
    smap = M.dof_map(L)
    xyz = M.slot_coords(L)
    np.testing.assert_allclose(xyz, rm.coords[smap], rtol=0, atol=1e-14)
    mass = M.lumped_mass(L)
    np.testing.assert_allclose(mass, omg.lumped_mass(rm)[smap], rtol=1e-13, atol=0)
    # copies of one vertex are bitwise equal
    order = np.argsort(smap, kind="stable")
    same = smap[order][1:] == smap[order][:-1]
    assert np.array_equal(xyz[order][1:][same], xyz[order][:-1][same])
    assert np.array_equal(mass[order][1:][same], mass[order][:-1][same])


@pytest.mark.parametrize("kx,ky,jit,L", [(1, 1, 0.0, 0), (1, 1, 0.0, 3), (3, 2, 0.15, 2), (4, 4, 0.15, 4)])
def test_p2_dof_map_matches_oracle(lib, kx, ky, jit, L):
    """The library's P2 global numbering and the oracle's name the same DoFs:
    one bijection between the two id sets maps every slot."""
    import oracle.p2 as p2
    from inputs import rect_mesh
    m = rect_mesh(kx, ky, jit, 0)
    M = lib.Mesh(m.coords, m.cells)
    pm = p2.P2Mesh(m.coords, m.cells, L)
    ns, ng = M.p2_num_slots(L)
    assert ng == pm.n_global
    assert ns == m.n_cells * oracle.p2_dofs_per_macro(L)
    mine, ref = M.p2_dof_map(L), pm.slot_map()
    assert mine.shape == ref.shape
    assert set(mine.tolist()) == set(range(ng))
    fwd = {}
    for a, b in zip(mine.tolist(), ref.tolist()):
        assert fwd.setdefault(a, b) == b
    assert len(set(fwd.values())) == ng
    # vertices keep the P1 numbering
    nv = oracle.slots_per_macro(2, L)
    per = oracle.p2_dofs_per_macro(L)
    vslots = np.concatenate([np.arange(c * per, c * per + nv) for c in range(m.n_cells)])
    np.testing.assert_array_equal(mine[vslots], M.dof_map(L))


def test_apply_batch_argument_checks_without_a_gpu(lib):
    """hyteg_apply_batch validates its arguments before touching the device:
    an empty batch is a no-op, a negative count or NULL arrays are EINVAL."""
    C = lib._capi
    n0 = C.lib.hyteg_apply_batch(None, None, lib.F64, None, None, 0, None)
    assert n0 == 0
    assert C.lib.hyteg_apply_batch(None, None, lib.F64, None, None, -1, None) == C.EINVAL
    assert C.lib.hyteg_apply_batch(None, None, lib.F64, None, None, 1, None) == C.EINVAL
    assert b"NULL" in C.lib.hyteg_last_error() or b"null" in C.lib.hyteg_last_error().lower()
