"""2D apply on the GPU against the oracle, element by element (needs a GPU)."""
import numpy as np
import pytest

from inputs import unit_square_mesh, random_vector, workload
import oracle
from parity import oracle_reference, check_close, gpu_apply, TOL

pytestmark = pytest.mark.gpu

KINDS = ["f64", "f32", "f64_ieee"]


def _lib():
    import paper_2305_15116_gb300 as H
    return H


@pytest.mark.parametrize("kind", KINDS)
def test_two_right_triangles_level7(cuda, kind):
    """Unit square as two macro-triangles at level 7, Dirichlet rows identity."""
    coarse, L, seed = workload("square2_L7")
    M = _lib().Mesh(coarse.coords, coarse.cells).refine(L)
    rm, x, y, absrow = oracle_reference(coarse, L, x_seed=seed, kind=kind)
    smap = M.dof_map(L)
    yg = gpu_apply(M, L, x[smap], kind)
    check_close(yg, y[smap], absrow[smap], kind, "square2_L7")


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("L", [0, 1, 2, 3, 5, 6, 7])
def test_jittered_32_macros(cuda, kind, L):
    """32 jittered macros; levels span no interior (L<=1), one partial strip
    (L=5: 30 interior columns), ragged strips and row chunks (L=6, 7)."""
    coarse = unit_square_mesh(4, 0.15, 0)
    M = _lib().Mesh(coarse.coords, coarse.cells).refine(L)
    rm, x, y, absrow = oracle_reference(coarse, L, x_seed=1, kind=kind)
    smap = M.dof_map(L)
    yg = gpu_apply(M, L, x[smap], kind)
    check_close(yg, y[smap], absrow[smap], kind, f"jit32 L{L}")


@pytest.mark.parametrize("kind", ["f64", "f32"])
def test_no_dirichlet_any_vertex_order(cuda, kind):
    """Plain stiffness (no boundary rows) on cells with permuted vertex order."""
    coarse = unit_square_mesh(3, 0.12, 9)
    rng = np.random.default_rng(5)
    cells = np.array([c[rng.permutation(3)] for c in coarse.cells])
    L = 6
    M = _lib().Mesh(coarse.coords, cells, bc=0).refine(L)

    class C:  # same coarse mesh with the permuted cells
        coords = coarse.coords
    C.cells = cells
    rm, x, y, absrow = oracle_reference(C, L, bc=False, x_seed=3, kind=kind)
    smap = M.dof_map(L)
    yg = gpu_apply(M, L, x[smap], kind)
    check_close(yg, y[smap], absrow[smap], kind, "permuted, no bc")


def test_deterministic_and_stream(cuda):
    import torch
    coarse = unit_square_mesh(4, 0.15, 0)
    L = 7
    M = _lib().Mesh(coarse.coords, coarse.cells).refine(L)
    ns, ng = M.num_slots(L)
    x = torch.from_numpy(random_vector(ng, 2)[M.dof_map(L)]).cuda()
    y1 = torch.empty_like(x)
    y2 = torch.empty_like(x)
    M.apply(L, x, y1)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        M.apply(L, x, y2, stream=s)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)


def test_errors(cuda):
    import torch
    H = _lib()
    coarse = unit_square_mesh(2, 0.1, 0)
    M = H.Mesh(coarse.coords, coarse.cells).refine(3)
    ns, _ = M.num_slots(3)
    x = torch.zeros(ns, dtype=torch.float64, device="cuda")
    with pytest.raises(H.HytegError) as e:
        M.apply(3, x, x)
    assert e.value.code == -1  # x and y overlap
    with pytest.raises(H.HytegError) as e:
        M.apply_raw(4, H.F64, x.data_ptr(), x.data_ptr() + 8 * ns, 0)
    assert e.value.code == -5  # level not refined
    with pytest.raises(H.HytegError) as e:
        M.apply_raw(3, 7, x.data_ptr(), x.data_ptr(), 0)
    assert e.value.code == -1


@pytest.mark.parametrize("kind", ["f64", "f32"])
def test_apply_host(cuda, kind):
    import torch
    coarse = unit_square_mesh(4, 0.15, 0)
    L = 6
    M = _lib().Mesh(coarse.coords, coarse.cells).refine(L)
    rm, x, y, absrow = oracle_reference(coarse, L, x_seed=4, kind=kind)
    smap = M.dof_map(L)
    dt = torch.float32 if kind == "f32" else torch.float64
    xh = torch.from_numpy(x[smap]).to(dt).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    M.apply_host(L, xh, yh)
    check_close(yh.double().numpy(), y[smap], absrow[smap], kind, "apply_host")


def _interface_slots(n, n_cells):
    """Slots on macro edges of every macro (rows y=0, column x=0, hypotenuse)."""
    S = (n + 1) * (n + 2) // 2
    ys = np.arange(n + 1)
    starts = ys * (n + 2) - ys * (ys + 1) // 2
    local = np.unique(np.concatenate([np.arange(n + 1), starts, starts + (n - ys)]))
    return (np.arange(n_cells)[:, None] * S + local[None, :]).ravel()


@pytest.mark.parametrize("kind", KINDS)
def test_full_size_sampled(cuda, kind):
    """32 jittered macros at level 11 (67M DoFs), the benchmark's launch: every
    slot written, copies equal, and sampled rows (interior and interface)
    against the oracle's row-by-row evaluation."""
    import torch
    coarse, L, seed = workload("square32jit_L11")
    M = _lib().Mesh(coarse.coords, coarse.cells).refine(L)
    ns, ng = M.num_slots(L)
    smap = M.dof_map(L)
    x = random_vector(ng, seed)
    if kind == "f32":
        x = x.astype(np.float32).astype(np.float64)
    yg = gpu_apply(M, L, x[smap], kind)
    assert np.all(np.isfinite(yg))
    # copies of a DoF hold one value
    order = np.argsort(smap, kind="stable")
    sm, yo = smap[order], yg[order]
    same = sm[1:] == sm[:-1]
    assert np.array_equal(yo[1:][same], yo[:-1][same])
    rm = oracle.RefinedMesh(coarse.coords, coarse.cells, L)
    rng = np.random.default_rng(17)
    iface = _interface_slots(rm.n, coarse.n_cells)
    slots = np.concatenate([rng.integers(0, ns, 300), rng.choice(iface, 200, replace=False)])
    gids = smap[slots]
    yref = oracle.row_apply(rm, gids, x)
    absrow = np.array([_absrow(rm, g, x) for g in gids])
    check_close(yg[slots], yref, absrow, kind, "L11 sampled")


def _tiles_2d(n, th, width=62):
    """The macro-interior tiles of a level as the library cuts them: strips of
    `width` written columns from x = 1 (32 lanes x two columns, the outermost
    two halo), rows chunked by th from y = 1."""
    out = []
    for x0 in range(1, n - 1, width):
        ymax = n - 1 - x0
        for y0 in range(1, ymax + 1, th):
            out.append((x0, y0, min(y0 + th, ymax + 1)))
    return out


@pytest.mark.parametrize("kind", KINDS)
def test_full_size_every_tile_stratified(cuda, kind):
    """Level 11 (67M DoFs), every tile of the launch's work list (the tile
    height the refinement's autotuner picked): the first and last row of the
    tile at its first and last written column, against the oracle's
    row-by-row evaluation.  The 32 macros share one tile list; tile i is
    checked in macro i mod 32, so every macro takes part."""
    coarse, L, seed = workload("square32jit_L11")
    M = _lib().Mesh(coarse.coords, coarse.cells).refine(L)
    ns, ng = M.num_slots(L)
    smap = M.dof_map(L)
    x = random_vector(ng, seed)
    if kind == "f32":
        x = x.astype(np.float32).astype(np.float64)
    yg = gpu_apply(M, L, x[smap], kind)
    n = 1 << L
    S = (n + 1) * (n + 2) // 2
    H = _lib()
    rows = M.autotune_choice(L, {"f64": H.F64, "f32": H.F32, "f64_ieee": H.F64_IEEE}[kind])
    assert rows in (8, 16, 32, 64)  # the level was autotuned
    pts = set()
    width = 62
    for i, (x0, y0, y1) in enumerate(_tiles_2d(n, rows, width)):
        m = i % coarse.n_cells
        for yy in (y0, y1 - 1):
            for xx in (x0, x0 + 1, min(x0 + width - 1, n - 1 - yy), min(x0 + width - 2, n - 1 - yy)):
                pts.add(m * S + yy * (n + 2) - yy * (yy + 1) // 2 + xx)
    slots = np.array(sorted(pts))
    rm = oracle.RefinedMesh(coarse.coords, coarse.cells, L)
    gids = smap[slots]
    yref = oracle.row_apply(rm, gids, x)
    absrow = np.array([_absrow(rm, g, x) for g in gids])
    check_close(yg[slots], yref, absrow, kind, f"L11 tile corners ({len(slots)} rows)")


@pytest.fixture(scope="module")
def level9_oracle():
    coarse, _, seed = workload("square32jit_L11", level=9)
    rm = oracle.RefinedMesh(coarse.coords, coarse.cells, 9)
    A = oracle.operator_matrix(rm)
    return coarse, rm, A, seed


@pytest.mark.parametrize("kind", KINDS)
def test_level9_element_wise(cuda, kind, level9_oracle):
    """The 32-macro workload at level 9 (4.2M DoFs), element by element: a
    level whose tiles are cut into 32-row chunks for the float64 kernels."""
    coarse, rm, A, seed = level9_oracle
    M = _lib().Mesh(coarse.coords, coarse.cells).refine(9)
    x = random_vector(rm.n_global, seed)
    if kind == "f32":
        x = x.astype(np.float32).astype(np.float64)
    smap = M.dof_map(9)
    yg = gpu_apply(M, 9, x[smap], kind)
    y = oracle.spmv(A, x)
    absrow = abs(A) @ np.abs(x)
    check_close(yg, y[smap], absrow[smap], kind, "L9 element-wise")


def test_tile_autotuner_choices(cuda):
    """Levels of at least 2^20 slots get an autotuned tile height per element
    type; smaller levels keep the default tiles (choice 0).  The level-9
    element-wise test above runs the autotuned lists."""
    H = _lib()
    coarse = unit_square_mesh(4, 0.15, 0)
    M = H.Mesh(coarse.coords, coarse.cells).refine(9)
    for L, tuned in ((6, False), (7, False), (8, True), (9, True)):  # 32 x 8,385 slots at level 7 < 2^20
        for dt in (H.F64, H.F32, H.F64_IEEE):
            c = M.autotune_choice(L, dt)
            assert (c in (8, 16, 32, 64)) if tuned else c == 0, (L, dt, c)
    M.close()


def _absrow(rm, g, x):
    """sum_j |a_gj x_j| from the oracle's micro-elements around g."""
    from oracle.assemble import _incidences, _macro_element_matrices
    from oracle.refine import element_offsets, in_region
    if rm.boundary[g]:
        return abs(x[g])
    row = {}
    for m, p in _incidences(rm, g):
        for off in element_offsets(rm.dim):
            for r in range(rm.dim + 1):
                verts = (p - off[r])[None, :] + off
                if not np.all(in_region(verts, rm.n)):
                    continue
                K = _macro_element_matrices(rm, m, verts[None])[0]
                gv = rm.local_to_global(m, verts)
                for j, v in zip(gv, K[r]):
                    row[j] = row.get(j, 0.0) + v
    return sum(abs(v * x[j]) for j, v in row.items())


def test_apply_host_batch_matches_single_applies(cuda):
    """The pipelined host-buffer batch gives bitwise the results of one apply
    per vector (distinct inputs, odd and even batch sizes)."""
    import torch
    import paper_2305_15116_gb300 as H
    from inputs import unit_square_mesh, random_vector
    m = unit_square_mesh(4, 0.15, 0)
    L = 6
    M = H.Mesh(m.coords, m.cells).refine(L)
    ns, ng = M.num_slots(L)
    smap = M.dof_map(L)
    for count in (1, 2, 5):
        xs = [torch.from_numpy(random_vector(ng, 40 + i)[smap]).pin_memory() for i in range(count)]
        ys = [torch.full((ns,), float("nan"), dtype=torch.float64).pin_memory() for _ in range(count)]
        M.apply_host_batch(L, xs, ys)
        for i in range(count):
            xd = xs[i].cuda()
            yd = torch.empty_like(xd)
            M.apply(L, xd, yd)
            torch.cuda.synchronize()
            assert torch.equal(yd.cpu(), ys[i])


@pytest.mark.parametrize("kind", KINDS)
def test_apply_batch_is_bitwise_the_single_applies(cuda, kind):
    """hyteg_apply_batch: 70 products (two launches of the batched 2D kernel)
    on meshes of 2, 8 and 32 macros at levels 0..7, vectors repeating a mesh,
    and 3D products in between; every output equals that product's own
    hyteg_apply bit for bit (outputs start as NaN)."""
    import torch
    from inputs import unit_cube_kuhn_mesh
    H = _lib()
    dt = torch.float32 if kind == "f32" else torch.float64
    ieee = kind == "f64_ieee"
    c2 = [unit_square_mesh(1, 0.0, 0), unit_square_mesh(2, 0.15, 1), unit_square_mesh(4, 0.15, 0)]
    m2 = [H.Mesh(c.coords, c.cells).refine(7) for c in c2]
    c3 = unit_cube_kuhn_mesh(1, 0.1, 0)
    m3 = H.Mesh(c3.coords, c3.cells).refine(3)
    rng = np.random.default_rng(5)
    meshes, levels = [], []
    for i in range(70):
        if i % 23 == 11:
            meshes.append(m3)
            levels.append(int(rng.integers(0, 4)))
        else:
            meshes.append(m2[int(rng.integers(0, 3))])
            levels.append(int(rng.integers(0, 8)))
    xs, ys, refs = [], [], []
    for i, (M, lev) in enumerate(zip(meshes, levels)):
        ns, _ = M.num_slots(lev)
        x = torch.from_numpy(random_vector(ns, 100 + i)).to("cuda", dt)
        xs.append(x)
        ys.append(torch.full_like(x, float("nan")))
        r = torch.full_like(x, float("nan"))
        M.apply(lev, x, r, ieee=ieee)
        refs.append(r)
    H.apply_batch(meshes, levels, xs, ys, ieee=ieee)
    torch.cuda.synchronize()
    for i in range(70):
        assert torch.equal(ys[i], refs[i]), (i, levels[i])


def test_apply_batch_errors(cuda):
    import torch
    H = _lib()
    coarse = unit_square_mesh(2, 0.1, 0)
    M = H.Mesh(coarse.coords, coarse.cells).refine(3)
    ns, _ = M.num_slots(3)
    x = torch.zeros(ns, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(H.HytegError) as e:
        H.apply_batch([M, M], [3, 3], [x, x], [y, x])
    assert e.value.code == -1  # x and y overlap in the second entry
    ns4, _ = M.num_slots(4)
    x4 = torch.zeros(ns4, dtype=torch.float64, device="cuda")
    with pytest.raises(H.HytegError) as e:
        H.apply_batch([M], [4], [x4], [torch.zeros_like(x4)])
    assert e.value.code == -5  # level not refined
    with pytest.raises(ValueError):
        H.apply_batch([M], [3, 3], [x], [y])
    assert H.apply_batch([], [], [], []) == []
