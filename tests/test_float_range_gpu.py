"""Applies on inputs far from magnitude 1, against the oracle (needs a GPU).

The float64 apply computes in float-float arithmetic (two fp32 parts), whose
exponent range is far narrower than float64's; inputs outside its range must
still give the float64 result (those rows are recomputed in native fp64).
These tests feed vectors scaled towards both ends of the float64 range, mixed
magnitudes in neighbouring DoFs, a few 1e300 entries, exact zeros of both
signs and float64 subnormals to the 2D, 3D and P2 applies in every element
type the type can represent, and compare every row with the oracle's float64
product.

Bound per row: |y - y_oracle| <= tol_row * sum_j |a_ij x_j|
+ 8 eps max_j |a_ij| sum_j |x_j| + 64 * (smallest subnormal of the element
type).  The second term covers the weights: the library forms each stencil
weight from its own element sums, which differ from the oracle's assembled
entries by a few ulps of the row's largest entry, and that difference only
shows when |x_j| varies over many orders of magnitude inside a row.  The last
term is the absolute rounding floor that gradual underflow gives any
floating-point evaluation of the row.
"""
import numpy as np
import pytest

import oracle
import oracle.p2 as p2
from inputs import unit_square_mesh, unit_cube_kuhn_mesh, range_vector
from parity import TOL, dtype_args

pytestmark = pytest.mark.gpu

F64_PATTERNS = ["scale:-100", "scale:-79", "scale:-72", "scale:64", "scale:65", "scale:125", "mixed", "huge",
                "sparse", "subnormal"]
F32_PATTERNS = ["scale:-100", "scale:-79", "scale:100", "mixed", "sparse"]
CASES = [(k, p) for k in ("f64", "f64_ieee") for p in F64_PATTERNS] + [("f32", p) for p in F32_PATTERNS]


def _lib():
    import paper_2305_15116_gb300 as H
    return H


def _floor(kind):
    return 64 * (2.0 ** -149 if kind == "f32" else 2.0 ** -1074)


EPS = 2.0 ** -53


def _terms(A, x):
    """Per row of the CSR matrix A: sum_j |a_ij x_j| and max_j |a_ij| sum_j |x_j|."""
    aa = abs(A).tocsr()
    pat = aa.copy()
    pat.data[:] = 1.0
    return aa @ np.abs(x), aa.max(axis=1).toarray().ravel() * (pat @ np.abs(x))


def _row_terms(rm, g, x):
    """The same two sums for one row g, from the oracle's micro-elements."""
    from oracle.assemble import _incidences, _macro_element_matrices
    from oracle.refine import element_offsets, in_region
    if rm.boundary[g]:
        return abs(x[g]), abs(x[g])
    row = {}
    for m, p in _incidences(rm, g):
        for off in element_offsets(rm.dim):
            for r in range(rm.dim + 1):
                verts = (p - off[r])[None, :] + off
                if not np.all(in_region(verts, rm.n)):
                    continue
                K = _macro_element_matrices(rm, m, verts[None])[0]
                for j, v in zip(rm.local_to_global(m, verts), K[r]):
                    row[j] = row.get(j, 0.0) + v
    wmax = max(abs(v) for v in row.values())
    return sum(abs(v * x[j]) for j, v in row.items()), wmax * sum(abs(x[j]) for j in row)


def _check(yg, yref, terms, kind, where):
    absrow, wx = terms
    tn, tr = TOL[kind]
    fl = _floor(kind)
    assert np.all(np.isfinite(yg)), f"{where}: non-finite output"
    d = np.abs(yg - yref)
    norm = np.abs(yref).max()
    assert d.max() <= tn * norm + fl, f"{where}: norm-wise error {d.max():.3e} vs {tn * norm:.3e}"
    bad = d > tr * absrow + 8 * EPS * wx + fl
    assert not bad.any(), (f"{where}: per-row bound broken at {np.nonzero(bad)[0][:5]}: "
                           f"{d[bad][:5]} vs {(tr * absrow)[bad][:5]}")


def _x(n, seed, pattern, kind):
    x = range_vector(n, seed, pattern)
    if kind == "f32":
        x = x.astype(np.float32).astype(np.float64)  # the fp32 apply sees fp32-rounded inputs
    return x


def _apply(M, L, xs_np, kind, p2_op=False):
    import torch
    dt, ieee = dtype_args(kind)
    xs = torch.from_numpy(xs_np).to("cuda", dt)
    ys = torch.full_like(xs, float("nan"))
    if p2_op:
        M.p2_apply(L, xs, ys, ieee=ieee)
    else:
        M.apply(L, xs, ys, ieee=ieee)
    torch.cuda.synchronize()
    return ys.double().cpu().numpy()


def _p1_case(coarse, L, kind, pattern, seed):
    M = _lib().Mesh(coarse.coords, coarse.cells).refine(L)
    rm = oracle.RefinedMesh(coarse.coords, coarse.cells, L)
    A = oracle.operator_matrix(rm)
    x = _x(rm.n_global, seed, pattern, kind)
    smap = M.dof_map(L)
    yg = _apply(M, L, x[smap], kind)
    t = _terms(A, x)
    _check(yg, (A @ x)[smap], (t[0][smap], t[1][smap]), kind, f"{coarse.name} L{L} {kind} {pattern}")


@pytest.mark.parametrize("kind,pattern", CASES)
def test_2d_range(cuda, kind, pattern):
    """32 jittered macro-triangles at level 6: macro-interior tiles (float-
    float rows and their native recomputation) and interface points."""
    _p1_case(unit_square_mesh(4, 0.15, 0), 6, kind, pattern, 11)


@pytest.mark.parametrize("kind,pattern", CASES)
def test_3d_range(cuda, kind, pattern):
    """48 jittered macro-tets at level 3 (slab kernel, interior units and
    boundary points) and one cube of 6 at level 5."""
    _p1_case(unit_cube_kuhn_mesh(2, 0.1, 0), 3, kind, pattern, 12)
    _p1_case(unit_cube_kuhn_mesh(1, 0.1, 1), 5, kind, pattern, 13)


@pytest.mark.parametrize("kind,pattern", [(k, p) for k in ("f64", "f64_ieee") for p in ("mixed", "scale:-100",
                                                                                       "huge")])
def test_3d_row_kernel_range_sampled(cuda, kind, pattern):
    """Level 7 (n = 128) runs the row kernel and its row-end companion:
    sampled rows against the oracle's row-by-row product."""
    coarse = unit_cube_kuhn_mesh(1, 0.1, 4)
    L = 7
    M = _lib().Mesh(coarse.coords, coarse.cells).refine(L)
    ns, ng = M.num_slots(L)
    smap = M.dof_map(L)
    x = _x(ng, 14, pattern, kind)
    yg = _apply(M, L, x[smap], kind)
    assert np.all(np.isfinite(yg))
    rm = oracle.RefinedMesh(coarse.coords, coarse.cells, L)
    rng = np.random.default_rng(37)
    slots = rng.integers(0, ns, 200)
    gids = smap[slots]
    yref = oracle.row_apply(rm, gids, x)
    t = np.array([_row_terms(rm, g, x) for g in gids])
    _check(yg[slots], yref, (t[:, 0], t[:, 1]), kind, f"3D L7 {kind} {pattern}")


@pytest.mark.parametrize("kind,pattern", CASES)
def test_p2_range(cuda, kind, pattern):
    """P2 (vertex + edge DoFs) on 8 jittered macro-triangles at level 5: row
    kernel, boundary kernel and the interface reductions."""
    coarse = unit_square_mesh(2, 0.15, 3)
    L = 5
    pm = p2.P2Mesh(coarse.coords, coarse.cells, L)
    A = pm.operator_matrix()
    x = _x(pm.n_global, 15, pattern, kind)
    M = _lib().Mesh(coarse.coords, coarse.cells).refine(L)
    smap = pm.slot_map()
    yg = _apply(M, L, x[smap], kind, p2_op=True)
    t = _terms(A, x)
    _check(yg, (A @ x)[smap], (t[0][smap], t[1][smap]), kind, f"P2 L{L} {kind} {pattern}")


@pytest.mark.parametrize("kind", ["f64", "f32"])
def test_batched_apply_range(cuda, kind):
    """The batched 2D launch shares the macro-interior code: mixed magnitudes
    through hyteg_apply_batch on two meshes."""
    import torch
    H = _lib()
    dt, _ = dtype_args(kind)
    meshes, levels, xs, ys, refs = [], [], [], [], []
    for k, L, seed in ((2, 5, 16), (4, 4, 17)):
        coarse = unit_square_mesh(k, 0.15, k)
        M = H.Mesh(coarse.coords, coarse.cells).refine(L)
        rm = oracle.RefinedMesh(coarse.coords, coarse.cells, L)
        A = oracle.operator_matrix(rm)
        x = _x(rm.n_global, seed, "mixed", kind)
        smap = M.dof_map(L)
        meshes.append(M)
        levels.append(L)
        xs.append(torch.from_numpy(x[smap]).to("cuda", dt))
        ys.append(torch.full_like(xs[-1], float("nan")))
        t = _terms(A, x)
        refs.append(((A @ x)[smap], (t[0][smap], t[1][smap])))
    H.apply_batch(meshes, levels, xs, ys)
    torch.cuda.synchronize()
    for i, (yr, ar) in enumerate(refs):
        _check(ys[i].double().cpu().numpy(), yr, ar, kind, f"batch entry {i}")


def test_weights_outside_the_float_float_range(cuda):
    """A mesh scaled by 2^-40 has 3D stencil weights of about 2^-44, whose
    largest lies below the float-float weight range: its float64 applies run
    the native fp64 kernels and still meet the float64 bound."""
    coarse = unit_cube_kuhn_mesh(1, 0.1, 2)

    class C:
        coords = np.ldexp(coarse.coords, -40)
        cells = coarse.cells
        name = "cube_scaled"
    _p1_case(C, 4, "f64", "scale:0", 18)
