"""The oracle's operator pinned to closed forms, invariants and brute force
(CPU only).  Each check is also run against deliberately broken variants of
the oracle's element matrix (planted on the CPU) to show that a plausible
mistake fails at least one pin."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import oracle.assemble as asm
from inputs import unit_square_mesh, unit_cube_kuhn_mesh, random_vector


def _mesh(dim, k, jit, seed=0):
    m = unit_square_mesh(k, jit, seed) if dim == 2 else unit_cube_kuhn_mesh(k, jit, seed)
    return m.coords, m.cells


# ---------------------------------------------------------------- pin checks
# Each returns None when the pin holds and raises AssertionError otherwise.

def pin_reference_elements(stiff):
    # textbook P1 element matrices of the reference triangle and tetrahedron
    K2 = stiff(np.eye(2))[0]
    np.testing.assert_allclose(K2, [[1, -0.5, -0.5], [-0.5, 0.5, 0], [-0.5, 0, 0.5]], atol=1e-15)
    K3 = stiff(np.eye(3))[0]
    ref3 = np.array([[3, -1, -1, -1], [-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]]) / 6
    np.testing.assert_allclose(K3, ref3, atol=1e-15)


def pin_five_point_2d(L=3):
    """Two right-isosceles macros: every non-boundary row is the 5-point
    [4, -1, -1, -1, -1] in physical directions, independent of L."""
    rm = oracle.RefinedMesh(*_mesh(2, 1, 0.0), L)
    A = oracle.operator_matrix(rm).tocsr()
    h = 1.0 / rm.n
    for i in np.nonzero(~rm.boundary)[0]:
        cols = A.indices[A.indptr[i]:A.indptr[i + 1]]
        vals = A.data[A.indptr[i]:A.indptr[i + 1]]
        got = {}
        for j, v in zip(cols, vals):
            if abs(v) > 1e-12:
                got[tuple(np.round((rm.coords[j] - rm.coords[i]) / h).astype(int))] = v
        want = {(0, 0): 4.0, (1, 0): -1.0, (-1, 0): -1.0, (0, 1): -1.0, (0, -1): -1.0}
        assert got.keys() == want.keys(), (i, got)
        for key in want:
            assert abs(got[key] - want[key]) < 1e-13, (i, key, got[key])


def pin_seven_point_3d(k=2, L=2):
    """Unjittered Kuhn cubes: the refined mesh is the Freudenthal triangulation
    of a uniform grid, whose P1 Laplacian row is h * [6, -1 x 6] with zero
    diagonal couplings."""
    rm = oracle.RefinedMesh(*_mesh(3, k, 0.0), L)
    A = oracle.operator_matrix(rm).tocsr()
    h = 1.0 / (k * rm.n)
    for i in np.nonzero(~rm.boundary)[0]:
        cols = A.indices[A.indptr[i]:A.indptr[i + 1]]
        vals = A.data[A.indptr[i]:A.indptr[i + 1]]
        got = {}
        for j, v in zip(cols, vals):
            if abs(v) > 1e-12 * h:
                got[tuple(np.round((rm.coords[j] - rm.coords[i]) / h).astype(int))] = v / h
        want = {(0, 0, 0): 6.0}
        for ax in range(3):
            for s in (-1, 1):
                e = [0, 0, 0]
                e[ax] = s
                want[tuple(e)] = -1.0
        assert got.keys() == want.keys(), (i, got)
        for key in want:
            assert abs(got[key] - want[key]) < 1e-12, (i, key, got[key])


def _angle(p, a, b):
    u, v = a - p, b - p
    return math.acos(float(u @ v) / (np.linalg.norm(u) * np.linalg.norm(v)))


def pin_cotangent_rows_2d(L=3):
    """Jittered macros: a macro-interior row is the cotangent stencil of the
    macro's angles th0, th1, th2 at v0, v1, v2: the neighbours along v1-v0
    couple with -cot th2, along v2-v0 with -cot th1, along v2-v1 with
    -cot th0, centre 2 (cot th0 + cot th1 + cot th2)."""
    rm = oracle.RefinedMesh(*_mesh(2, 4, 0.15, 3), L)
    A = oracle.operator_matrix(rm).tocsr()
    n = rm.n
    for m in range(rm.cells.shape[0]):
        v = rm.coarse_coords[rm.cells[m]]
        c0 = 1 / math.tan(_angle(v[0], v[1], v[2]))
        c1 = 1 / math.tan(_angle(v[1], v[2], v[0]))
        c2 = 1 / math.tan(_angle(v[2], v[0], v[1]))
        want = {(0, 0): 2 * (c0 + c1 + c2), (1, 0): -c2, (-1, 0): -c2, (0, 1): -c1, (0, -1): -c1,
                (1, -1): -c0, (-1, 1): -c0}
        for y in range(1, n - 1):
            for x in range(1, n - y):
                i = rm.local_to_global(m, np.array([[x, y]]))[0]
                for (dx, dy), w in want.items():
                    j = rm.local_to_global(m, np.array([[x + dx, y + dy]]))[0]
                    assert abs(A[i, j] - w) < 1e-12 * max(1, abs(w)), (m, x, y, dx, dy, A[i, j], w)
                assert abs(A[i].sum()) < 1e-12


def pin_invariants(dim, k, jit, L, seed=1):
    """Zero row sums and symmetry of the stiffness; Dirichlet rows identity;
    A (linear) = 0 at non-boundary rows; energy of a linear function equals
    |Omega| |grad u|^2 = |grad u|^2 on the unit box; PSD."""
    rm = oracle.RefinedMesh(*_mesh(dim, k, jit, seed), L)
    K = oracle.assemble_stiffness(rm)
    assert abs(K - K.T).max() < 1e-12
    assert np.abs(np.asarray(K.sum(axis=1))).max() < 1e-11
    A = oracle.operator_matrix(rm)
    b = rm.boundary
    Ab = A[np.nonzero(b)[0]]
    assert abs(Ab - sp.eye(rm.n_global, format="csr")[np.nonzero(b)[0]]).max() == 0.0
    g = np.arange(1, dim + 1, dtype=np.float64) * 0.7
    u = rm.coords @ g + 0.3
    r = oracle.spmv(A, u)
    assert np.abs(r[~b]).max() < 1e-11
    np.testing.assert_allclose(r[b], u[b], rtol=0, atol=0)
    energy = u @ oracle.spmv(K, u)
    assert abs(energy - g @ g) < 1e-11 * (g @ g)


def pin_quadratic_energy_converges(dim, jit):
    """Energy of the interpolant of q = |x|^2 tends to int |grad q|^2 = 4 d/3
    with error O(h^2) (ratio ~4 per level)."""
    exact = 4.0 * dim / 3.0
    errs = []
    levels = [1, 2, 3, 4] if dim == 2 else [0, 1, 2]
    k = 2 if dim == 2 else 1
    for L in levels:
        rm = oracle.RefinedMesh(*_mesh(dim, k, jit, 5), L)
        K = oracle.assemble_stiffness(rm)
        u = (rm.coords ** 2).sum(axis=1)
        errs.append(abs(u @ oracle.spmv(K, u) - exact))
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.0 < r < 5.5 for r in ratios[1:]), (errs, ratios)


ALL_PINS = [
    ("reference_elements", lambda: pin_reference_elements(oracle.element_stiffness)),
    ("five_point_2d", pin_five_point_2d),
    ("seven_point_3d", pin_seven_point_3d),
    ("cotangent_rows_2d", pin_cotangent_rows_2d),
    ("invariants_2d", lambda: pin_invariants(2, 4, 0.15, 3)),
    ("invariants_3d", lambda: pin_invariants(3, 2, 0.1, 2)),
    ("quadratic_2d", lambda: pin_quadratic_energy_converges(2, 0.15)),
    ("quadratic_3d", lambda: pin_quadratic_energy_converges(3, 0.0)),
]


@pytest.mark.parametrize("name,check", ALL_PINS, ids=[p[0] for p in ALL_PINS])
def test_pin(name, check):
    check()


def test_psd_and_constant_nullspace():
    for dim, k, L in [(2, 2, 1), (3, 1, 1)]:
        rm = oracle.RefinedMesh(*_mesh(dim, k, 0.1), L)
        K = oracle.assemble_stiffness(rm).toarray()
        ev = np.linalg.eigvalsh(K)
        assert ev.min() > -1e-12
        assert (np.abs(ev) < 1e-10).sum() == 1


@pytest.mark.parametrize("dim,k,jit,L", [(2, 2, 0.15, 3), (3, 1, 0.1, 2), (3, 2, 0.1, 1)])
def test_row_apply_matches_assembled(dim, k, jit, L):
    rm = oracle.RefinedMesh(*_mesh(dim, k, jit, 7), L)
    A = oracle.operator_matrix(rm)
    x = random_vector(rm.n_global, 11)
    y = oracle.spmv(A, x)
    gids = np.arange(rm.n_global)
    y1 = oracle.row_apply(rm, gids, x)
    np.testing.assert_allclose(y1, y, rtol=0, atol=1e-13)


# ------------------------------------------------------- planted mistakes
# Each mutant of the element matrix must fail at least one pin.

def _sign_slip(J):
    J = np.asarray(J, dtype=np.float64)
    J = J[None] if J.ndim == 2 else J
    k, d, _ = J.shape
    vol = np.abs(np.linalg.det(J)) / math.factorial(d)
    JinvT = np.transpose(np.linalg.inv(J), (0, 2, 1))
    G = np.empty((k, d, d + 1))
    G[:, :, 1:] = JinvT
    G[:, :, 0] = +JinvT.sum(axis=2)  # wrong sign
    return vol[:, None, None] * np.einsum("kai,kaj->kij", G, G)


def _transposed(J):
    J = np.asarray(J, dtype=np.float64)
    J = J[None] if J.ndim == 2 else J
    return oracle.element_stiffness(np.transpose(J, (0, 2, 1)))


def _no_volume(J):
    J = np.asarray(J, dtype=np.float64)
    J = J[None] if J.ndim == 2 else J
    d = J.shape[1]
    vol = np.abs(np.linalg.det(J)) / math.factorial(d)
    return oracle.element_stiffness(J) / vol[:, None, None]


def _no_factorial(J):
    J = np.asarray(J, dtype=np.float64)
    J = J[None] if J.ndim == 2 else J
    d = J.shape[1]
    return oracle.element_stiffness(J) * math.factorial(d)


@pytest.mark.parametrize("mutant", [_sign_slip, _transposed, _no_volume, _no_factorial])
def test_planted_mistakes_fail_a_pin(mutant, monkeypatch):
    monkeypatch.setattr(asm, "element_stiffness", mutant)
    failed = []
    for name, check in ALL_PINS:
        if name == "reference_elements":
            try:
                pin_reference_elements(mutant)
            except AssertionError:
                failed.append(name)
            continue
        try:
            check()
        except AssertionError:
            failed.append(name)
    assert failed, f"mutant {mutant.__name__} passed every pin"
