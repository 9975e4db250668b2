"""The oracle's multigrid pieces pinned to identities of nested P1 spaces and
to closed forms (CPU only)."""
import numpy as np
import pytest

import oracle
import oracle.multigrid as mg
from inputs import unit_square_mesh, unit_cube_kuhn_mesh


def _mesh(dim, k, jit, seed=0):
    m = unit_square_mesh(k, jit, seed) if dim == 2 else unit_cube_kuhn_mesh(k, jit, seed)
    return m.coords, m.cells


def pin_galerkin(dim, k, jit, L, prolong=mg.prolongation):
    """Nested P1 spaces: P^T K_l P = K_{l-1} (stiffness without boundary rows)."""
    meshes = [oracle.RefinedMesh(*_mesh(dim, k, jit), l) for l in range(L + 1)]
    for l in range(1, L + 1):
        P = prolong(meshes[l], meshes[l - 1])
        Kf = oracle.assemble_stiffness(meshes[l])
        Kc = oracle.assemble_stiffness(meshes[l - 1])
        G = (P.T @ Kf @ P - Kc).toarray()
        assert np.abs(G).max() < 1e-12 * max(1.0, np.abs(Kc.toarray()).max()), (l, np.abs(G).max())


def pin_prolongation_linear(dim, k, jit, L, prolong=mg.prolongation):
    """P interpolates linear functions exactly and its rows sum to one."""
    c = oracle.RefinedMesh(*_mesh(dim, k, jit), L - 1)
    f = oracle.RefinedMesh(*_mesh(dim, k, jit), L)
    P = prolong(f, c)
    g = np.arange(1, dim + 1) * 0.37
    np.testing.assert_allclose(P @ (c.coords @ g + 0.2), f.coords @ g + 0.2, atol=1e-14)
    np.testing.assert_allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0, atol=1e-15)


@pytest.mark.parametrize("dim,k,jit,L", [(2, 4, 0.15, 4), (2, 1, 0.0, 3), (3, 2, 0.1, 2), (3, 1, 0.0, 3)])
def test_galerkin_identity(dim, k, jit, L):
    pin_galerkin(dim, k, jit, L)


@pytest.mark.parametrize("dim,k,jit,L", [(2, 4, 0.15, 3), (3, 2, 0.1, 2)])
def test_prolongation_linear(dim, k, jit, L):
    pin_prolongation_linear(dim, k, jit, L)


def test_lumped_mass_closed_forms():
    # total mass = |Omega| = 1 on the unit square and cube, any jitter
    for dim, k, jit, L in [(2, 4, 0.15, 3), (3, 2, 0.1, 2)]:
        rm = oracle.RefinedMesh(*_mesh(dim, k, jit), L)
        assert abs(mg.lumped_mass(rm).sum() - 1.0) < 1e-13
    # uniform right triangles: an interior vertex owns 6 triangles of area h^2/2
    rm = oracle.RefinedMesh(*_mesh(2, 1, 0.0), 4)
    h = 1.0 / rm.n
    m = mg.lumped_mass(rm)
    np.testing.assert_allclose(m[~rm.boundary], h * h, rtol=1e-13)
    # Kuhn cubes: an interior vertex owns 24 tets of volume h^3/6
    rm3 = oracle.RefinedMesh(*_mesh(3, 1, 0.0), 3)
    h3 = 1.0 / rm3.n
    np.testing.assert_allclose(mg.lumped_mass(rm3)[~rm3.boundary], h3 ** 3, rtol=1e-13)


@pytest.mark.parametrize("dim,k,jit,L", [(2, 4, 0.15, 5), (3, 2, 0.1, 3)])
def test_vcycle_converges_to_1e10(dim, k, jit, L):
    H = mg.Hierarchy(*_mesh(dim, k, jit), L)
    rm = H.meshes[L]
    f = np.prod(np.sin(np.pi * rm.coords), axis=1) + 0.1 * np.random.default_rng(2).standard_normal(rm.n_global)
    b = mg.poisson_rhs(rm, f)
    u, hist = H.solve(b, rtol=1e-10)
    rates = [hist[i + 1] / hist[i] for i in range(1, len(hist) - 1)]
    assert hist[-1] <= 1e-10
    assert max(rates) < 0.5, rates
    # the returned u solves the system: check with an independent product
    r = b - oracle.spmv(H.A[L], u)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)


def test_manufactured_solution_second_order():
    """-Lap u = 2 pi^2 sin(pi x) sin(pi y): nodal error falls ~4x per level."""
    errs = []
    for L in (3, 4, 5):
        H = mg.Hierarchy(*_mesh(2, 2, 0.1), L)
        rm = H.meshes[L]
        x, y = rm.coords[:, 0], rm.coords[:, 1]
        b = mg.poisson_rhs(rm, 2 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y))
        u, _ = H.solve(b, rtol=1e-12)
        errs.append(np.abs(u - np.sin(np.pi * x) * np.sin(np.pi * y)).max())
    assert 3.0 < errs[0] / errs[1] < 5.5 and 3.0 < errs[1] / errs[2] < 5.5, errs


def _bad_prolongation(fine, coarse):
    """A plausible slip: midpoints weighted 0.4 / 0.6 instead of 1/2."""
    P = mg.prolongation(fine, coarse).tocoo()
    v = P.data.copy()
    half = v == 0.5
    idx = np.nonzero(half)[0]
    v[idx[0::2]] = 0.4
    v[idx[1::2]] = 0.6
    import scipy.sparse as sp
    return sp.csr_matrix((v, (P.row, P.col)), shape=P.shape)


def test_planted_prolongation_mistake_fails_a_pin():
    failed = 0
    for pin in (pin_galerkin, pin_prolongation_linear):
        try:
            pin(2, 4, 0.15, 3, prolong=_bad_prolongation)
        except AssertionError:
            failed += 1
    assert failed >= 1


def test_float64_residual_floor_and_two_part_iterate():
    """The relative residual a float64 solution can reach is bounded below by
    the rounding of its entries: fl(u*) has residual A (u* - fl(u*)).  On the
    32-macro solve workload (f = sin(pi x) sin(pi y) + 0.1 N(0,1), lumped
    mass) at levels 4..6 that floor, computed with an exactly rounded
    residual, matches the estimate from independent half-ulp errors within
    5 %, grows 4x per level (h^-2), and extrapolates to about 1.9e-10 at level
    10 — above an rtol of 1e-10.  An iterate of two float64 parts (iterative
    refinement on the exact residual, the correction's rounding error kept in
    the low part) reaches a relative residual below 1e-12 at every level,
    and a tenth of the floor."""
    from oracle.multigrid import (Hierarchy, poisson_rhs, relres_exact, float64_floor_estimate,
                                  solve_two_part)
    from inputs import workload, random_normal
    floors = []
    for L in (4, 5, 6):
        coarse, _, seed = workload("square32jit_L10_solve", level=L)
        h = Hierarchy(coarse.coords, coarse.cells, L)
        rm = h.meshes[L]
        xy = rm.coords
        f = np.sin(np.pi * xy[:, 0]) * np.sin(np.pi * xy[:, 1]) + 0.1 * random_normal(rm.n_global, seed)
        b = poisson_rhs(rm, f)
        inter = ~rm.boundary
        u_hi, u_lo = solve_two_part(h, b, 40)
        dd = relres_exact(h.A[L], b, (u_hi, u_lo), inter)
        floor = relres_exact(h.A[L], b, (u_hi,), inter)  # u_hi = fl(u_hi + u_lo)
        assert dd < 1e-12 and dd < 0.1 * floor, (L, dd, floor)
        est = float64_floor_estimate(h.A[L], b, u_hi, inter)
        assert abs(floor / est - 1.0) < 0.05, (L, floor, est)
        floors.append(floor)
    for a, c in zip(floors, floors[1:]):
        assert 3.5 < c / a < 4.5, floors
    at10 = floors[-1] * 4.0 ** 4
    assert 1.2e-10 < at10 < 3e-10, at10
