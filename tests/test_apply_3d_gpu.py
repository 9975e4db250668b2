"""3D apply (15-point stencil on Kuhn-refined macro-tets) on the GPU against
the oracle, element by element (needs a GPU)."""
import numpy as np
import pytest

from inputs import unit_cube_kuhn_mesh, random_vector, workload
import oracle
from parity import oracle_reference, check_close, gpu_apply
from test_apply_2d_gpu import _absrow

pytestmark = pytest.mark.gpu

KINDS = ["f64", "f32", "f64_ieee"]


def _lib():
    import paper_2305_15116_gb300 as H
    return H


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("k,L", [(1, 0), (1, 1), (1, 2), (2, 2), (2, 3), (1, 4), (1, 5)])
def test_jittered_cubes(cuda, kind, k, L):
    """Levels 0-1 have no macro interior, 2 has one interior point per macro,
    4-5 have ragged strips (n-2-z not a multiple of 30)."""
    coarse = unit_cube_kuhn_mesh(k, 0.1, 0)
    M = _lib().Mesh(coarse.coords, coarse.cells).refine(L)
    rm, x, y, absrow = oracle_reference(coarse, L, x_seed=1, kind=kind)
    smap = M.dof_map(L)
    yg = gpu_apply(M, L, x[smap], kind)
    check_close(yg, y[smap], absrow[smap], kind, f"cube k{k} L{L}")


@pytest.mark.parametrize("kind", ["f64", "f32"])
def test_permuted_vertex_order_no_bc(cuda, kind):
    coarse = unit_cube_kuhn_mesh(1, 0.0, 0)
    rng = np.random.default_rng(8)
    cells = np.array([c[rng.permutation(4)] for c in coarse.cells])

    class C:
        coords = coarse.coords
    C.cells = cells
    L = 4
    M = _lib().Mesh(C.coords, cells, bc=0).refine(L)
    rm, x, y, absrow = oracle_reference(C, L, bc=False, x_seed=2, kind=kind)
    smap = M.dof_map(L)
    yg = gpu_apply(M, L, x[smap], kind)
    check_close(yg, y[smap], absrow[smap], kind, "3d permuted")


@pytest.mark.parametrize("kind", KINDS)
def test_full_size_sampled(cuda, kind):
    """384 jittered macro-tets at level 6 (17M DoFs), the benchmark's launch."""
    coarse, L, seed = workload("cube384jit_L6")
    M = _lib().Mesh(coarse.coords, coarse.cells).refine(L)
    ns, ng = M.num_slots(L)
    smap = M.dof_map(L)
    x = random_vector(ng, seed)
    if kind == "f32":
        x = x.astype(np.float32).astype(np.float64)
    yg = gpu_apply(M, L, x[smap], kind)
    assert np.all(np.isfinite(yg))
    order = np.argsort(smap, kind="stable")
    sm, yo = smap[order], yg[order]
    same = sm[1:] == sm[:-1]
    assert np.array_equal(yo[1:][same], yo[:-1][same])
    rm = oracle.RefinedMesh(coarse.coords, coarse.cells, L)
    rng = np.random.default_rng(23)
    slots = rng.integers(0, ns, 400)
    gids = smap[slots]
    yref = oracle.row_apply(rm, gids, x)
    absrow = np.array([_absrow(rm, g, x) for g in gids])
    check_close(yg[slots], yref, absrow, kind, "L6 3D sampled")


@pytest.mark.parametrize("kind", ["f64", "f32"])
def test_level7_row_kernel_sampled(cuda, kind):
    """Level 7 (n = 128) is above the shared-memory slab kernel's limit and runs
    the row-sweep kernel with the stencil interface step: sampled rows."""
    coarse = unit_cube_kuhn_mesh(1, 0.1, 4)
    L = 7
    M = _lib().Mesh(coarse.coords, coarse.cells).refine(L)
    ns, ng = M.num_slots(L)
    smap = M.dof_map(L)
    x = random_vector(ng, 6)
    if kind == "f32":
        x = x.astype(np.float32).astype(np.float64)
    yg = gpu_apply(M, L, x[smap], kind)
    assert np.all(np.isfinite(yg))
    rm = oracle.RefinedMesh(coarse.coords, coarse.cells, L)
    rng = np.random.default_rng(29)
    slots = rng.integers(0, ns, 300)
    gids = smap[slots]
    yref = oracle.row_apply(rm, gids, x)
    absrow = np.array([_absrow(rm, g, x) for g in gids])
    check_close(yg[slots], yref, absrow, kind, "3D L7 sampled")


def test_slab_autotune_choices_and_parity(cuda):
    """Refinement autotunes the slab kernel's work split on 3D levels of at
    least 2^20 slots; every element type's chosen list must still cover every
    slot (outputs start as NaN) and match the oracle on sampled rows."""
    H = _lib()
    coarse = unit_cube_kuhn_mesh(2, 0.1, 3)  # 48 macro-tets
    M = H.Mesh(coarse.coords, coarse.cells).refine(6)
    for L, tuned in ((4, False), (5, False), (6, True)):
        for dt in (H.F64, H.F32, H.F64_IEEE):
            c = M.autotune_choice(L, dt)
            assert (c in (2, 3, 4, 5, 6, 8)) if tuned else c == 0, (L, dt, c)
    L = 6
    ns, ng = M.num_slots(L)
    smap = M.dof_map(L)
    rm = oracle.RefinedMesh(coarse.coords, coarse.cells, L)
    rng = np.random.default_rng(31)
    slots = rng.integers(0, ns, 200)
    gids = smap[slots]
    for kind in KINDS:
        x = random_vector(ng, 8)
        if kind == "f32":
            x = x.astype(np.float32).astype(np.float64)
        yg = gpu_apply(M, L, x[smap], kind)
        assert np.all(np.isfinite(yg)), kind
        yref = oracle.row_apply(rm, gids, x)
        absrow = np.array([_absrow(rm, g, x) for g in gids])
        check_close(yg[slots], yref, absrow, kind, f"autotuned 3D L6 {kind}")
