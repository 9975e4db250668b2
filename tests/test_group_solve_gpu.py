"""Solves of several problems in lockstep (hyteg_solve_two_part_group; needs
a GPU): every solve step is one launch for all problems still iterating.
Each problem's iterations, relative residual and solution are bitwise those
of the same problem solved alone, and the oracle's float64 product confirms
the residuals."""
import numpy as np
import pytest

import oracle
from inputs import rect_mesh, box_kuhn_mesh, unit_square_mesh

pytestmark = pytest.mark.gpu


def _lib():
    import paper_2305_15116_gb300 as H
    return H


def _problem(coarse, L, seed, scale=0.0):
    import torch
    H = _lib()
    c = coarse if scale == 0.0 else type("C", (), {"coords": np.ldexp(coarse.coords, int(scale)),
                                                   "cells": coarse.cells})
    M = H.Mesh(c.coords, c.cells).refine(L).solver_setup(L)
    ns, _ = M.num_slots(L)
    b = torch.empty(ns, dtype=torch.float64, device="cuda")
    M.poisson_rhs(L, seed, 0.1, b)
    return M, b


def _alone(M, L, b, mode, rtol=1e-10):
    import torch
    u, lo = torch.zeros_like(b), torch.zeros_like(b)
    it, rel = M.solve_two_part(L, b, u, lo, mode=mode, rtol=rtol, max_iter=100)
    torch.cuda.synchronize()
    return it, rel, u.cpu().numpy(), lo.cpu().numpy()


def _group(Ms, L, bs, mode, rtol=1e-10):
    import torch
    H = _lib()
    us = [torch.zeros_like(b) for b in bs]
    los = [torch.zeros_like(b) for b in bs]
    res = H.solve_two_part_group(Ms, L, bs, us, los, mode=mode, rtol=rtol, max_iter=100)
    torch.cuda.synchronize()
    return [(it, rel, u.cpu().numpy(), lo.cpu().numpy()) for (it, rel), u, lo in zip(res, us, los)]


CASES = {
    # 2D: three meshes of 8, 12 and 32 macro-triangles, level 6
    "2d": (lambda: [rect_mesh(2, 2, 0.15, 0), rect_mesh(2, 3, 0.15, 1), unit_square_mesh(4, 0.15, 2)], 6),
    # 3D: 6, 12 and 48 macro-tets, level 4 (the slab kernel)
    "3d": (lambda: [box_kuhn_mesh(1, 1, 1, 0.1, 0), box_kuhn_mesh(2, 1, 1, 0.1, 1), box_kuhn_mesh(2, 2, 2, 0.1, 2)],
           4),
}


@pytest.mark.parametrize("mode", ["mixed", "f64"])
@pytest.mark.parametrize("case", ["2d", "3d"])
def test_group_is_bitwise_the_solves_alone(cuda, case, mode):
    H = _lib()
    code = H.SOLVE_MIXED if mode == "mixed" else H.SOLVE_F64
    meshes, L = CASES[case]
    probs = [_problem(c, L, 40 + i) for i, c in enumerate(meshes())]
    alone = [_alone(M, L, b, code) for M, b in probs]
    # fresh meshes for the group (its workspaces start as a first solve's)
    gprobs = [_problem(c, L, 40 + i) for i, c in enumerate(meshes())]
    grouped = _group([M for M, _ in gprobs], L, [b for _, b in gprobs], code)
    for i, (a, g) in enumerate(zip(alone, grouped)):
        assert a[0] == g[0] and a[1] == g[1], (i, a[:2], g[:2])
        assert a[1] <= 1e-10
        assert np.array_equal(a[2], g[2]) and np.array_equal(a[3], g[3]), i
    # the oracle confirms every residual
    for c, (M, b), (it, rel, u, lo) in zip(meshes(), gprobs, grouped):
        smap = M.dof_map(L)
        rm = oracle.RefinedMesh(c.coords, c.cells, L)
        A = oracle.operator_matrix(rm)
        bg = np.zeros(rm.n_global)
        bg[smap] = b.cpu().numpy()
        ug = np.zeros(rm.n_global)
        ug[smap] = u
        r = bg - oracle.spmv(A, ug)
        assert np.linalg.norm(r) <= 2e-10 * np.linalg.norm(bg)
    for M, _ in probs + gprobs:
        M.close()


def test_group_with_levels_outside_the_float_float_range(cuda):
    """A 3D group whose second mesh is scaled by 2^-40, so that its stencil
    weights (about 2^-40) fail the float-float weight check: the group's
    float-float applies split by element type (native fp64 for that mesh)
    and every result stays that of the solve alone."""
    H = _lib()
    L = 3
    cs = [box_kuhn_mesh(1, 1, 1, 0.1, 3), box_kuhn_mesh(1, 1, 1, 0.1, 4), box_kuhn_mesh(2, 1, 1, 0.1, 5)]
    scales = [0.0, -40.0, 0.0]
    alone = []
    for i, (c, sc) in enumerate(zip(cs, scales)):
        M, b = _problem(c, L, 60 + i, sc)
        alone.append(_alone(M, L, b, H.SOLVE_F64, rtol=1e-9))
        M.close()
    gp = [_problem(c, L, 60 + i, sc) for i, (c, sc) in enumerate(zip(cs, scales))]
    grouped = _group([M for M, _ in gp], L, [b for _, b in gp], H.SOLVE_F64, rtol=1e-9)
    for a, g in zip(alone, grouped):
        assert a[1] <= 1e-9
        assert a[0] == g[0] and a[1] == g[1]
        assert np.array_equal(a[2], g[2]) and np.array_equal(a[3], g[3])
    for M, _ in gp:
        M.close()


def test_group_arguments(cuda):
    import torch
    H = _lib()
    M2, b2 = _problem(rect_mesh(1, 1, 0.0, 0), 3, 1)
    M3, b3 = _problem(box_kuhn_mesh(1, 1, 1, 0.0, 0), 3, 2)
    z = lambda b: torch.zeros_like(b)
    with pytest.raises(H.HytegError):  # dimensions differ
        H.solve_two_part_group([M2, M3], 3, [b2, b3], [z(b2), z(b3)], [z(b2), z(b3)])
    with pytest.raises(H.HytegError):  # one mesh twice
        H.solve_two_part_group([M2, M2], 3, [b2, b2], [z(b2), z(b2)], [z(b2), z(b2)])
    u = z(b2)
    with pytest.raises(H.HytegError):  # u_lo == u
        H.solve_two_part_group([M2], 3, [b2], [u], [u])
    assert H.solve_two_part_group([], 3, [], [], []) == []
    M2.close()
    M3.close()


def test_group_larger_than_one_launch(cuda):
    """18 problems: every solve step needs two launches of at most 16 meshes
    each (the group launch's parameter block); each result stays bitwise
    that of its solve alone."""
    H = _lib()
    L = 4
    cs = [rect_mesh(1 + k % 3, 1 + (k // 3) % 2, 0.15, k) for k in range(18)]
    alone = []
    for i, c in enumerate(cs):
        M, b = _problem(c, L, 80 + i)
        alone.append(_alone(M, L, b, H.SOLVE_MIXED))
        M.close()
    gp = [_problem(c, L, 80 + i) for i, c in enumerate(cs)]
    grouped = _group([M for M, _ in gp], L, [b for _, b in gp], H.SOLVE_MIXED)
    for a, g in zip(alone, grouped):
        assert a[1] <= 1e-10
        assert a[0] == g[0] and a[1] == g[1]
        assert np.array_equal(a[2], g[2]) and np.array_equal(a[3], g[3])
    for M, _ in gp:
        M.close()


def test_group_above_the_slab_levels_runs_one_after_another(cuda):
    """3D level 7 (the row kernel, no group launch): the group call solves
    its problems one after another, each exactly as alone."""
    H = _lib()
    L = 7
    cs = [box_kuhn_mesh(1, 1, 1, 0.1, 5), box_kuhn_mesh(1, 1, 1, 0.1, 6)]
    alone = []
    for i, c in enumerate(cs):
        M, b = _problem(c, L, 90 + i)
        alone.append(_alone(M, L, b, H.SOLVE_MIXED, rtol=1e-9))
        M.close()
    gp = [_problem(c, L, 90 + i) for i, c in enumerate(cs)]
    grouped = _group([M for M, _ in gp], L, [b for _, b in gp], H.SOLVE_MIXED, rtol=1e-9)
    for a, g in zip(alone, grouped):
        assert a[1] <= 1e-9
        assert a[0] == g[0] and a[1] == g[1]
        assert np.array_equal(a[2], g[2]) and np.array_equal(a[3], g[3])
    for M, _ in gp:
        M.close()
