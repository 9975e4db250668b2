"""Multigrid on the GPU against the oracle's textbook V-cycle (needs a GPU)."""
import numpy as np
import pytest

import oracle
import oracle.multigrid as omg
from inputs import unit_square_mesh, unit_cube_kuhn_mesh, random_vector

pytestmark = pytest.mark.gpu


def _lib():
    import paper_2305_15116_gb300 as H
    return H


def _coarse(dim):
    return unit_square_mesh(4, 0.15, 0) if dim == 2 else unit_cube_kuhn_mesh(2, 0.1, 0)


def _setup(dim, L):
    c = _coarse(dim)
    M = _lib().Mesh(c.coords, c.cells).refine(L).solver_setup(L)
    H = omg.Hierarchy(c.coords, c.cells, L)
    return c, M, H


def _dev(a, dt):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


@pytest.mark.parametrize("kind", ["f64", "f32"])
@pytest.mark.parametrize("dim,L", [(2, 1), (2, 3), (2, 5), (3, 1), (3, 3)])
def test_restrict_and_prolong(cuda, dim, L, kind):
    import torch
    dt = torch.float64 if kind == "f64" else torch.float32
    tol = 1e-13 if kind == "f64" else 2e-6
    c, M, H = _setup(dim, L)
    for lf in range(1, L + 1):
        sf, sc = M.dof_map(lf), M.dof_map(lf - 1)
        rf = random_vector(H.meshes[lf].n_global, 10 + lf)
        ref = H.P[lf].T @ rf
        ref[H.meshes[lf - 1].boundary] = 0.0
        bc = torch.full((len(sc),), float("nan"), dtype=dt, device="cuda")
        M.restrict(lf, _dev(rf[sf], dt), bc)
        got = bc.double().cpu().numpy()
        assert np.all(np.isfinite(got))
        np.testing.assert_allclose(got, ref[sc], rtol=0, atol=tol * np.abs(ref).max())
        ec = random_vector(H.meshes[lf - 1].n_global, 20 + lf)
        uf0 = random_vector(H.meshes[lf].n_global, 30 + lf)
        uf = _dev(uf0[sf], dt)
        M.prolong_add(lf, _dev(ec[sc], dt), uf)
        want = uf0 + H.P[lf] @ ec
        np.testing.assert_allclose(uf.double().cpu().numpy(), want[sf], rtol=0, atol=tol * np.abs(want).max())


def _rhs(H, L, seed=2):
    rm = H.meshes[L]
    f = np.prod(np.sin(np.pi * rm.coords), axis=1) + 0.1 * np.random.default_rng(seed).standard_normal(rm.n_global)
    return omg.poisson_rhs(rm, f)


@pytest.mark.parametrize("kind", ["f64", "f32"])
@pytest.mark.parametrize("dim,L", [(2, 2), (2, 5), (3, 3), (3, 4)])
def test_one_vcycle_matches_oracle(cuda, dim, L, kind):
    import torch
    dt = torch.float64 if kind == "f64" else torch.float32
    c, M, H = _setup(dim, L)
    b = _rhs(H, L)
    smap = M.dof_map(L)
    u = torch.zeros(len(smap), dtype=dt, device="cuda")
    M.vcycle(L, _dev(b[smap], dt), u)
    ref = H.vcycle(L, np.zeros_like(b), b)
    got = u.double().cpu().numpy()
    tol = 1e-11 if kind == "f64" else 2e-5
    np.testing.assert_allclose(got, ref[smap], rtol=0, atol=tol * np.abs(ref).max())


@pytest.mark.parametrize("mode", ["mixed", "f64"])
@pytest.mark.parametrize("dim,L", [(2, 6), (3, 3)])
def test_solve_reaches_1e10(cuda, dim, L, mode):
    import torch
    Hh = _lib()
    c, M, H = _setup(dim, L)
    b = _rhs(H, L, seed=5)
    smap = M.dof_map(L)
    bd = _dev(b[smap], torch.float64)
    u = torch.zeros_like(bd)
    it, rel = M.solve(L, bd, u, mode=Hh.SOLVE_MIXED if mode == "mixed" else Hh.SOLVE_F64, rtol=1e-10, max_iter=60)
    assert rel <= 1e-10 and it < 60
    us = u.cpu().numpy()
    # copies of a DoF agree
    order = np.argsort(smap, kind="stable")
    same = smap[order][1:] == smap[order][:-1]
    assert np.array_equal(us[order][1:][same], us[order][:-1][same])
    # the oracle's float64 product confirms the residual
    ug = np.zeros(H.meshes[L].n_global)
    ug[smap] = us
    r = b - oracle.spmv(H.A[L], ug)
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b)
    # and the solution agrees with the oracle's multigrid solution
    uo, _ = H.solve(b, rtol=1e-12)
    assert np.abs(ug - uo).max() <= 1e-8 * np.abs(uo).max()


@pytest.mark.parametrize("mode", ["mixed", "f64"])
def test_two_part_solve_below_the_float64_floor(cuda, mode):
    """hyteg_solve_two_part on 32 right-isosceles macro-triangles at level 7:
    their stencil weights (4, -1, 0) are exact in binary, so the library's
    operator and the oracle's assembled matrix agree bitwise and the oracle's
    exactly rounded residual can confirm the two-part solution below the
    floor that a float64 iterate cannot pass (about 3e-12 at this level; the
    oracle measures it on u, the float64 rounding of u + u_lo).  On jittered
    meshes the two operators differ by a few ulps of their entries, which
    shows in the residual at the size of that same floor."""
    import torch
    Hh = _lib()
    c = unit_square_mesh(4, 0.0, 0)
    L = 7
    M = Hh.Mesh(c.coords, c.cells).refine(L).solver_setup(L)
    H = omg.Hierarchy(c.coords, c.cells, L)
    b = _rhs(H, L, seed=6)
    smap = M.dof_map(L)
    bd = _dev(b[smap], torch.float64)
    u = torch.zeros_like(bd)
    ulo = torch.zeros_like(bd)
    it, rel = M.solve_two_part(L, bd, u, ulo, mode=Hh.SOLVE_MIXED if mode == "mixed" else Hh.SOLVE_F64,
                               rtol=1e-12, max_iter=80)
    assert rel <= 1e-12 and it < 80, (it, rel)
    us, ls = u.cpu().numpy(), ulo.cpu().numpy()
    order = np.argsort(smap, kind="stable")
    same = smap[order][1:] == smap[order][:-1]
    assert np.array_equal(us[order][1:][same], us[order][:-1][same])
    assert np.array_equal(ls[order][1:][same], ls[order][:-1][same])
    n = H.meshes[L].n_global
    ug, lg = np.zeros(n), np.zeros(n)
    ug[smap], lg[smap] = us, ls
    assert np.all(np.abs(lg) <= np.spacing(np.abs(ug)))  # u is the float64 rounding of u + u_lo
    inter = ~H.meshes[L].boundary
    exact = omg.relres_exact(H.A[L], b, (ug, lg), inter)
    assert exact <= 1.05e-12 and abs(exact - rel) <= 0.05 * exact + 1e-15, (exact, rel)
    floor = omg.relres_exact(H.A[L], b, (ug,), inter)
    est = omg.float64_floor_estimate(H.A[L], b, ug, inter)
    assert 0.5 * est < floor < 2.0 * est and floor > 2.0 * exact, (floor, est, exact)


@pytest.mark.parametrize("mode", ["mixed", "f64"])
@pytest.mark.parametrize("dim,L", [(2, 6), (3, 4)])
def test_two_part_solve_jittered(cuda, dim, L, mode):
    """The two-part solve on jittered meshes reaches 1e-12 on the library's
    operator; copies agree, u is the float64 rounding of u + u_lo, and the
    oracle's float64 product confirms the residual to the level at which
    the two operators' entries differ."""
    import torch
    Hh = _lib()
    c, M, H = _setup(dim, L)
    b = _rhs(H, L, seed=7)
    smap = M.dof_map(L)
    bd = _dev(b[smap], torch.float64)
    u = torch.zeros_like(bd)
    ulo = torch.zeros_like(bd)
    it, rel = M.solve_two_part(L, bd, u, ulo, mode=Hh.SOLVE_MIXED if mode == "mixed" else Hh.SOLVE_F64,
                               rtol=1e-12, max_iter=80)
    assert rel <= 1e-12 and it < 80, (it, rel)
    us, ls = u.cpu().numpy(), ulo.cpu().numpy()
    order = np.argsort(smap, kind="stable")
    same = smap[order][1:] == smap[order][:-1]
    assert np.array_equal(us[order][1:][same], us[order][:-1][same])
    n = H.meshes[L].n_global
    ug, lg = np.zeros(n), np.zeros(n)
    ug[smap], lg[smap] = us, ls
    assert np.all(np.abs(lg) <= np.spacing(np.abs(ug)))
    inter = ~H.meshes[L].boundary
    exact = omg.relres_exact(H.A[L], b, (ug, lg), inter)
    est = omg.float64_floor_estimate(H.A[L], b, ug, inter)
    assert exact <= 1e-12 + 4.0 * est, (exact, est)
