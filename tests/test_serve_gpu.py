"""The Poisson model problem on the device (right-hand side, global gather)
and the solve server, against the oracle (needs a GPU)."""
import numpy as np
import pytest

import oracle
import oracle.multigrid as omg
from inputs import rect_mesh, box_kuhn_mesh, random_vector
from inputs.philox import philox_normal

pytestmark = pytest.mark.gpu


def _lib():
    import paper_2305_15116_gb300 as H
    return H


def _oracle_rhs(coarse, L, seed, noise):
    rm = oracle.RefinedMesh(coarse.coords, coarse.cells, L)
    f = np.prod(np.sin(np.pi * rm.coords), axis=1) + noise * philox_normal(np.arange(rm.n_global), seed)
    return rm, omg.poisson_rhs(rm, f)


CASES = [(rect_mesh(3, 2, 0.15, 4), 4), (rect_mesh(4, 4, 0.15, 0), 5), (box_kuhn_mesh(2, 1, 1, 0.1, 2), 3),
         (box_kuhn_mesh(2, 2, 2, 0.1, 0), 4)]


@pytest.mark.parametrize("coarse,L", CASES, ids=lambda v: getattr(v, "name", str(v)))
def test_poisson_rhs_and_gather(cuda, coarse, L):
    import torch
    H = _lib()
    M = H.Mesh(coarse.coords, coarse.cells).refine(L).solver_setup(L)
    ns, ng = M.num_slots(L)
    smap = M.dof_map(L)
    b = torch.full((ns,), float("nan"), dtype=torch.float64, device="cuda")
    M.poisson_rhs(L, 77, 0.1, b)
    bg = torch.full((ng,), float("nan"), dtype=torch.float64, device="cuda")
    M.to_global(L, b, bg)
    torch.cuda.synchronize()
    bs, bgh = b.cpu().numpy(), bg.cpu().numpy()
    assert np.all(np.isfinite(bgh))
    # every copy of a DoF holds the same bits, and the gather picks them
    assert np.array_equal(bgh[smap], bs)
    rm, ref = _oracle_rhs(coarse, L, 77, 0.1)
    np.testing.assert_allclose(bgh, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    assert np.all(bgh[rm.boundary] == 0.0)
    # the gather of an arbitrary consistent vector is exact
    v = random_vector(ng, 5)
    vs = torch.from_numpy(v[smap]).cuda()
    M.to_global(L, vs, bg)
    torch.cuda.synchronize()
    assert np.array_equal(bg.cpu().numpy(), v)


def _solve_oracle(coarse, L, b):
    H = omg.Hierarchy(coarse.coords, coarse.cells, L)
    u, _ = H.solve(b, rtol=1e-12)
    return H, u


def _server(cap=8 << 30, workers=3):
    return _lib().Server(cap, workers)


@pytest.mark.parametrize("mode", ["mixed", "f64"])
def test_server_solves_match_oracle(cuda, mode):
    H = _lib()
    reqs = [(rect_mesh(4, 4, 0.15, 0), 5, 11), (rect_mesh(3, 2, 0.15, 4), 4, 12), (box_kuhn_mesh(2, 2, 2, 0.1, 0), 3, 13)]
    with _server() as sv:
        out = []
        for coarse, L, seed in reqs:
            rm = oracle.RefinedMesh(coarse.coords, coarse.cells, L)
            u = np.full(rm.n_global, np.nan)
            b = np.full(rm.n_global, np.nan)
            t = sv.submit(coarse.coords, coarse.cells, L, seed, 0.1,
                          mode=H.SOLVE_MIXED if mode == "mixed" else H.SOLVE_F64, rtol=1e-9, max_iter=60,
                          u_out=u, b_out=b)
            assert t is not None
            out.append((t, coarse, L, seed, u, b))
        for t, coarse, L, seed, u, b in out:
            r = sv.wait(t, 300)
            assert r is not None and r.status == H.REQ_DONE, r
            assert r.relres <= 1e-9 and r.iters < 60
            assert r.n_global == u.size
            _, bref = _oracle_rhs(coarse, L, seed, 0.1)
            np.testing.assert_allclose(b, bref, rtol=0, atol=1e-13 * np.abs(bref).max())
            Hh, uref = _solve_oracle(coarse, L, bref)
            res = bref - oracle.spmv(Hh.A[L], u)
            assert np.linalg.norm(res) <= 1.01e-9 * np.linalg.norm(bref)
            assert np.abs(u - uref).max() <= 1e-7 * np.abs(uref).max()
            sv.release(t)


def test_server_batch_is_bitwise_equal_to_alone(cuda):
    H = _lib()
    probe = (rect_mesh(4, 4, 0.15, 0), 6, 21)
    others = [(rect_mesh(2, 3, 0.15, 1), 5, 22), (box_kuhn_mesh(2, 2, 2, 0.1, 0), 4, 23),
              (rect_mesh(4, 4, 0.15, 0), 6, 24), (box_kuhn_mesh(1, 2, 2, 0.1, 3), 3, 25)]

    def run(batch):
        with _server(workers=4) as sv:
            res = []
            for coarse, L, seed in batch:
                n = oracle.RefinedMesh(coarse.coords, coarse.cells, L).n_global
                u = np.full(n, np.nan)
                res.append((sv.submit(coarse.coords, coarse.cells, L, seed, 0.1, rtol=1e-9, u_out=u), u))
            for t, _ in res:
                assert sv.wait(t, 300).status == H.REQ_DONE
            return [u for _, u in res]

    alone = run([probe])[0]
    batched = run(others[:2] + [probe] + others[2:])[2]
    assert np.array_equal(alone, batched)


def test_server_cache_and_stats(cuda):
    H = _lib()
    coarse = rect_mesh(3, 3, 0.15, 7)
    with _server(workers=1) as sv:
        t1 = sv.submit(coarse.coords, coarse.cells, 5, 1, 0.1)
        r1 = sv.wait(t1, 300)
        t2 = sv.submit(coarse.coords, coarse.cells, 5, 2, 0.1)
        r2 = sv.wait(t2, 300)
        assert r1.status == r2.status == H.REQ_DONE
        assert not r1.cache_hit and r2.cache_hit
        s = sv.stats()
        assert s["done"] == 2 and s["failed"] == 0 and s["cache_hits"] == 1 and s["cached_meshes"] == 1
        assert s["in_flight"] == 0 and s["reserved_bytes"] == 0 and s["arena_used"] > 0


def test_server_admission_and_errors(cuda):
    H = _lib()
    big = rect_mesh(4, 4, 0.15, 0)
    # the estimate of a level-9 request on 32 macros is ~0.45 GB: one fits in
    # 0.7 GB, two do not
    with _server(cap=700 << 20, workers=1) as sv:
        # larger than the whole cap: refused for good
        with pytest.raises(H.HytegError) as ei:
            sv.submit(big.coords, big.cells, 11, 1)
        assert ei.value.code == -1
        # bad arguments
        with pytest.raises(H.HytegError):
            sv.submit(big.coords, big.cells, 0, 1)
        with pytest.raises(H.HytegError):
            sv.submit(big.coords, big.cells, 5, 1, rtol=0.0)
        # the second of two such requests waits for the first
        t1 = sv.submit(big.coords, big.cells, 9, 1, rtol=1e-9)
        assert t1 is not None
        t2 = sv.submit(big.coords, big.cells, 9, 2, rtol=1e-9)
        if t2 is None:  # refused while the first is in flight
            r1 = sv.wait(t1, 300)
            assert r1.status == H.REQ_DONE
            t2 = sv.submit(big.coords, big.cells, 9, 2, rtol=1e-9)
            assert t2 is not None
        else:  # the first had already finished
            assert sv.poll(t1).finished
        assert sv.wait(t2, 300).status == H.REQ_DONE
        # a zero timeout on a fresh request reports "not finished" or the result
        t3 = sv.submit(big.coords, big.cells, 9, 3, rtol=1e-9)
        r3 = sv.wait(t3, 0.0)
        assert r3 is None or r3.finished
        if r3 is None:
            with pytest.raises(H.HytegError) as ei:
                sv.release(t3)  # not finished
            assert ei.value.code == -5
        with pytest.raises(H.HytegError):
            sv.release(123456789)  # unknown ticket
        assert sv.wait(t3, 300).status == H.REQ_DONE
        # a degenerate coarse mesh fails inside the server with the mesh error
        bad = big.coords.copy()
        bad[big.cells[0, 1]] = bad[big.cells[0, 0]]
        t4 = sv.submit(bad, big.cells, 3, 1)
        r4 = sv.wait(t4, 300)
        assert r4.status == H.REQ_FAILED and r4.error == -4


def test_server_wait_times_out_deterministically(cuda):
    """One worker: a request queued behind a long one (a level-10 solve on
    32 macros, which takes far longer than a millisecond to build and solve)
    cannot finish within 1 ms: the bounded wait reports HYTEG_ETIMEDOUT and
    the request is still queued."""
    H = _lib()
    big, small = rect_mesh(4, 4, 0.15, 0), rect_mesh(2, 1, 0.15, 1)
    with _server(workers=1) as sv:
        t1 = sv.submit(big.coords, big.cells, 10, 1, 0.1, rtol=1e-9)
        t2 = sv.submit(small.coords, small.cells, 4, 2, 0.1, rtol=1e-9)
        assert t1 is not None and t2 is not None
        assert sv.wait(t2, 0.001) is None  # HYTEG_ETIMEDOUT
        assert sv.poll(t2).status == H.REQ_QUEUED
        with pytest.raises(H.HytegError) as ei:
            sv.release(t2)  # not finished
        assert ei.value.code == -5
        assert sv.wait(t1, 300).status == H.REQ_DONE
        assert sv.wait(t2, 300).status == H.REQ_DONE


def test_server_allocation_failure_is_reported(cuda):
    """A device allocation that fails inside the server (injected on the host:
    the arena refuses the next allocation) fails that request with
    HYTEG_ENOMEM at once; the server keeps serving the next request."""
    H = _lib()
    coarse = rect_mesh(3, 2, 0.15, 4)
    with _server(workers=1) as sv:
        sv.inject_alloc_failures(1)
        t1 = sv.submit(coarse.coords, coarse.cells, 5, 1, 0.1, rtol=1e-9)
        r1 = sv.wait(t1, 300)
        assert r1.status == H.REQ_FAILED and r1.error == -2, r1
        assert "arena" in r1.message
        t2 = sv.submit(coarse.coords, coarse.cells, 5, 2, 0.1, rtol=1e-9)
        r2 = sv.wait(t2, 300)
        assert r2.status == H.REQ_DONE and r2.relres <= 1e-9
        s = sv.stats()
        assert s["failed"] == 1 and s["done"] == 1


@pytest.mark.parametrize("dim", [2, 3])
def test_server_groups_requests_of_one_class(cuda, dim):
    """One worker busy with a long request while five requests of one class
    queue up: the worker then solves them as one group (one launch per solve
    step for all), and every solution is bitwise that of the request solved
    alone."""
    H = _lib()
    if dim == 2:
        blocker = (rect_mesh(4, 4, 0.15, 9), 9, 30)
        same = [(rect_mesh(2, 2, 0.15, k), 6, 31 + k) for k in range(3)] + \
               [(rect_mesh(3, 2, 0.15, 5), 6, 35), (rect_mesh(2, 2, 0.15, 0), 6, 36)]
    else:
        blocker = (box_kuhn_mesh(2, 2, 2, 0.1, 9), 6, 30)
        same = [(box_kuhn_mesh(1, 1, 1, 0.1, k), 4, 31 + k) for k in range(3)] + \
               [(box_kuhn_mesh(2, 1, 1, 0.1, 5), 4, 35), (box_kuhn_mesh(1, 1, 1, 0.1, 0), 4, 36)]

    def n_of(coarse, L):
        return oracle.RefinedMesh(coarse.coords, coarse.cells, L).n_global

    alone = []
    with _server(workers=1) as sv:
        for coarse, L, seed in same:
            u = np.full(n_of(coarse, L), np.nan)
            lo = np.full_like(u, np.nan)
            t = sv.submit(coarse.coords, coarse.cells, L, seed, 0.1, rtol=1e-10, u_out=u, u_lo_out=lo)
            r = sv.wait(t, 300)
            assert r.status == H.REQ_DONE and r.group == 1
            alone.append((u, lo, r.iters, r.relres))
            sv.release(t)
    with _server(workers=1) as sv:
        c, L, seed = blocker
        tb = sv.submit(c.coords, c.cells, L, seed, 0.1, rtol=1e-10)
        outs = []
        for coarse, L, seed in same:
            u = np.full(n_of(coarse, L), np.nan)
            lo = np.full_like(u, np.nan)
            outs.append((sv.submit(coarse.coords, coarse.cells, L, seed, 0.1, rtol=1e-10, u_out=u, u_lo_out=lo), u, lo))
        assert sv.wait(tb, 300).status == H.REQ_DONE
        groups = []
        for (t, u, lo), (ua, loa, it, rel) in zip(outs, alone):
            r = sv.wait(t, 300)
            assert r.status == H.REQ_DONE
            groups.append(r.group)
            assert r.iters == it and r.relres == rel and rel <= 1e-10
            assert np.array_equal(u, ua) and np.array_equal(lo, loa)
        st = sv.stats()
    # the five queued behind the blocker: one group of five
    assert max(groups) >= 2 and st["group_solves"] >= 1 and st["grouped"] >= 2, (groups, st)
