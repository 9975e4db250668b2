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


def _z_cuts(n, chunks):
    """z-ranges of one macro-tet in the slab kernel's work list: a cut is
    placed after the slice at which the running count of slice points first
    reaches c/chunks of the macro's points, c = 1..chunks-1."""
    S = (n + 1) * (n + 2) * (n + 3) // 6
    cuts, acc = [0], 0
    for z in range(n + 1):
        m = n + 1 - z
        acc += m * (m + 1) // 2
        if len(cuts) < chunks and acc * chunks >= S * len(cuts) and z < n:
            cuts.append(z + 1)
    return cuts + [n + 1]


def _tet_slot(n, x, y, z):
    """Position of micro-vertex (x, y, z) in a macro's slot block: slices
    z = 0..n, each a triangle of rows y, each row x = 0..n-z-y."""
    N = n + 1
    b = N - z
    zs = N * (N + 1) * (N + 2) // 6 - b * (b + 1) * (b + 2) // 6
    return zs + y * b - y * (y - 1) // 2 + x


@pytest.mark.parametrize("kind", KINDS)
def test_full_size_every_z_range_edge(cuda, kind):
    """The benchmark's launch (384 jittered macro-tets, level 6) with the
    work split the refinement's autotuner chose for this element type: the
    first and last slice of every z-range, at the start and end of its first
    row and at its last row, in the first and last macro and six others."""
    coarse, L, seed = workload("cube384jit_L6")
    H = _lib()
    M = H.Mesh(coarse.coords, coarse.cells).refine(L)
    code = {"f64": H.F64, "f32": H.F32, "f64_ieee": H.F64_IEEE}[kind]
    chunks = M.autotune_choice(L, code) or 2
    n = 1 << L
    cuts = _z_cuts(n, chunks)
    assert len(cuts) == chunks + 1 and all(a < b for a, b in zip(cuts, cuts[1:]))
    ns, ng = M.num_slots(L)
    S = ns // coarse.n_cells
    assert S == (n + 1) * (n + 2) * (n + 3) // 6
    smap = M.dof_map(L)
    x = random_vector(ng, seed)
    if kind == "f32":
        x = x.astype(np.float32).astype(np.float64)
    yg = gpu_apply(M, L, x[smap], kind)
    assert np.all(np.isfinite(yg))
    rng = np.random.default_rng(41)
    cells = [0, coarse.n_cells - 1] + list(rng.choice(np.arange(1, coarse.n_cells - 1), 6, replace=False))
    slots = []
    for c in cells:
        for z0, z1 in zip(cuts, cuts[1:]):
            for z in sorted({z0, z1 - 1}):
                w = n - z  # the slice's rows y = 0..w, row y has x = 0..w-y
                pts = {(0, 0), (w, 0), (0, w)} if w < 2 else {(1, 1), (w - 2, 1), (1, w - 2), (0, 0), (w, 0)}
                slots += [c * S + _tet_slot(n, px, py, z) for px, py in pts]
    slots = np.unique(slots)
    rm = oracle.RefinedMesh(coarse.coords, coarse.cells, L)
    gids = smap[slots]
    yref = oracle.row_apply(rm, gids, x)
    absrow = np.array([_absrow(rm, g, x) for g in gids])
    check_close(yg[slots], yref, absrow, kind, f"L6 3D z-range edges ({chunks} per macro) {kind}")
