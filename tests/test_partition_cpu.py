"""The apply over macros partitioned across processes, host side, on the CPU
with gloo ranks (world sizes 2 and 3): every rank computes the partial rows
of its own cells — here from the oracle's per-macro element matrices, standing
in for hyteg_apply_partial on a GPU — exchanges the partials of shared DoFs
and sums every interface DoF in ascending macro order.  The ranks' results,
put together, are bitwise the single-rank result of the same partials, and
agree with the oracle's assembled operator."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = {
    "square8_L3": ("unit_square_mesh", (2, 0.15, 0), 3),
    "box12_L2": ("box_kuhn_mesh", (2, 1, 1, 0.1, 2), 2),
}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _coarse(case):
    import inputs
    fn, args, L = CASES[case]
    return getattr(inputs, fn)(*args), L


def _partials(coarse, L, c0, c1):
    """partial(x, y): every slot of cells c0..c1-1 gets its own macro's row
    (the oracle's stiffness of that macro alone applied to x)."""
    import oracle
    mats = []
    for c in range(c0, c1):
        rm = oracle.RefinedMesh(coarse.coords, coarse.cells[[c]], L)
        mats.append((oracle.assemble_stiffness(rm), rm.slot_map()))

    def partial(x, y):
        S = mats[0][1].size if mats else 0
        xs = x.numpy()
        out = y.numpy()
        for i, (K, smap) in enumerate(mats):
            xg = np.zeros(K.shape[0])
            xg[smap] = xs[i * S:(i + 1) * S]
            out[i * S:(i + 1) * S] = (K @ xg)[smap]
    return partial


def _x(coarse, L):
    import oracle
    from inputs import random_vector
    rm = oracle.RefinedMesh(coarse.coords, coarse.cells, L)
    x = random_vector(rm.n_global, 5)
    return rm, x, x[rm.slot_map()]


def _worker(rank, world, port, case, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2305_15116_gb300.partition import PartitionedApply, cell_blocks
        coarse, L = _coarse(case)
        rm, x, xs = _x(coarse, L)
        c0, c1 = cell_blocks(coarse.n_cells, world)[rank]
        S = xs.size // coarse.n_cells
        pa = PartitionedApply(coarse.coords, coarse.cells, L, rank, world, partial_apply=_partials(coarse, L, c0, c1))
        xl = torch.from_numpy(xs[c0 * S:c1 * S].copy())
        yl = torch.full_like(xl, float("nan"))
        pa.apply(xl, yl)
        q.put((rank, yl.numpy().copy()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case,world", [("square8_L3", 2), ("square8_L3", 3), ("box12_L2", 2)])
def test_partitioned_apply_is_bitwise_the_single_rank_apply(case, world):
    import torch
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2305_15116_gb300.partition import PartitionedApply
    coarse, L = _coarse(case)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    y_dist = np.concatenate([got[r] for r in range(world)])
    # one rank, the same partials: no exchange
    rm, x, xs = _x(coarse, L)
    one = PartitionedApply(coarse.coords, coarse.cells, L, 0, 1, partial_apply=_partials(coarse, L, 0, coarse.n_cells))
    y1 = torch.full((xs.size,), float("nan"), dtype=torch.float64)
    one.apply(torch.from_numpy(xs.copy()), y1)
    assert np.array_equal(y_dist, y1.numpy())
    # and the operator: the oracle's assembled matrix with Dirichlet rows
    A = oracle.operator_matrix(rm)
    ref = (A @ x)[rm.slot_map()]
    absrow = (abs(A) @ np.abs(x))[rm.slot_map()]
    assert np.all(np.abs(y_dist - ref) <= 1e-14 * absrow + 1e-300)


def test_plan_exchanges_only_shared_copies():
    """What a rank sends to a peer is exactly what the peer expects from it
    (the same global slots, ascending), every received copy belongs to a DoF
    the receiver holds, and no DoF of a single rank is exchanged."""
    sys.path.insert(0, ROOT)
    from paper_2305_15116_gb300.partition import PartitionPlan
    coarse, L = _coarse("square8_L3")
    world = 3
    plans = [PartitionPlan(coarse.coords, coarse.cells, L, r, world) for r in range(world)]
    S = plans[0].S
    import oracle
    gid = oracle.RefinedMesh(coarse.coords, coarse.cells, L).slot_map()
    for r, p in enumerate(plans):
        mine = set(gid[p.blocks[r][0] * S:p.blocks[r][1] * S])
        for peer in range(world):
            if peer == r:
                continue
            rcv = p.recv_slots.get(peer, np.zeros(0, np.int64))
            snd = plans[peer].send_slots.get(r, np.zeros(0, np.int64)) + plans[peer].blocks[peer][0] * S
            assert np.array_equal(rcv, snd)
            assert np.all(np.diff(rcv) > 0)
            assert all(g in mine for g in gid[rcv])


@pytest.mark.parametrize("case,world", [("square8_L3", 3), ("box12_L2", 2)])
def test_rank_mesh_has_the_whole_meshs_slot_layout(case, world):
    """Every rank's own mesh (its cells over the vertices they use) lays out
    its slots like the whole mesh's block of those cells: two slots of the
    rank's mesh hold the same DoF exactly when the whole mesh's slots do."""
    sys.path.insert(0, ROOT)
    from paper_2305_15116_gb300 import Mesh, BC_NONE
    from paper_2305_15116_gb300.partition import PartitionPlan
    coarse, L = _coarse(case)
    g = Mesh(coarse.coords, coarse.cells)
    gid = g.dof_map(L)
    g.close()
    for r in range(world):
        p = PartitionPlan(coarse.coords, coarse.cells, L, r, world)
        m = Mesh(p.coords, p.local_cells, BC_NONE)
        lid = m.dof_map(L)
        m.close()
        c0, c1 = p.blocks[r]
        blk = gid[c0 * p.S:c1 * p.S]
        assert lid.size == blk.size
        # the same partition of slots into DoFs: slot -> DoF is one to one
        # between the two numberings
        pairs = np.unique(np.stack([lid, blk]), axis=1).shape[1]
        assert pairs == np.unique(lid).size == np.unique(blk).size


def test_plan_arguments():
    """A rank outside the world, or more ranks than coarse cells (every rank
    owns at least one macro), are refused before any mesh is built."""
    sys.path.insert(0, ROOT)
    from paper_2305_15116_gb300.partition import PartitionPlan
    coarse, L = _coarse("square8_L3")
    with pytest.raises(ValueError):
        PartitionPlan(coarse.coords, coarse.cells, L, 3, 3)
    with pytest.raises(ValueError):
        PartitionPlan(coarse.coords, coarse.cells, L, 0, coarse.cells.shape[0] + 1)
