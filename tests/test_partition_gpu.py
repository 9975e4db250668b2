"""The partitioned apply with the library's partial rows on the GPU (needs a
GPU).  One process plays every rank of the partition: each rank refines a
mesh of its own block of cells and runs hyteg_apply_partial, the partials of
shared DoFs are handed from the senders' to the receivers' buffers (what the
communicator does between processes), and every rank completes its DoFs.
The ranks' results, put together, are bitwise hyteg_apply on the whole mesh,
in every element type."""
import numpy as np
import pytest

from inputs import unit_square_mesh, unit_cube_kuhn_mesh, random_vector

pytestmark = pytest.mark.gpu


def _lib():
    import paper_2305_15116_gb300 as H
    return H


def _partitioned(coarse, L, world, xs, kind):
    import torch
    from paper_2305_15116_gb300.partition import PartitionedApply
    ranks = [PartitionedApply(coarse.coords, coarse.cells, L, r, world) for r in range(world)]
    S = ranks[0].plan.S
    dt = torch.float32 if kind == "f32" else torch.float64
    xl, yl, sends, recvs = [], [], [], []
    for r, pa in enumerate(ranks):
        c0, c1 = pa.plan.blocks[r]
        xl.append(torch.from_numpy(xs[c0 * S:c1 * S].copy()).to("cuda", dt))
        yl.append(torch.full_like(xl[-1], float("nan")))
        sends.append(pa.begin(xl[-1], yl[-1], ieee=kind == "f64_ieee"))
        recvs.append(pa.receive_buffers(yl[-1]))
    for r in range(world):  # the exchange
        for peer, buf in recvs[r].items():
            buf.copy_(sends[peer][r])
    for r, pa in enumerate(ranks):
        pa.complete(xl[r], yl[r], recvs[r])
    torch.cuda.synchronize()
    out = np.concatenate([y.double().cpu().numpy() for y in yl])
    for pa in ranks:
        pa.close()
    return out


@pytest.mark.parametrize("kind", ["f64", "f64_ieee", "f32"])
@pytest.mark.parametrize("dim,world,L", [(2, 2, 6), (2, 3, 6), (3, 2, 4), (3, 4, 4), (3, 2, 7)])
def test_partitioned_apply_bitwise_on_gpu(cuda, dim, world, L, kind):
    """2D and 3D (level 4: the slab kernel; level 7: the row kernel), two to
    four ranks."""
    import torch
    H = _lib()
    if dim == 2:
        coarse = unit_square_mesh(4, 0.15, 0)
    else:
        coarse = unit_cube_kuhn_mesh(2, 0.1, 0) if L < 7 else unit_cube_kuhn_mesh(1, 0.1, 0)
    M = H.Mesh(coarse.coords, coarse.cells).refine(L)
    ns, ng = M.num_slots(L)
    xs = random_vector(ng, 9)[M.dof_map(L)]
    if kind == "f32":
        xs = xs.astype(np.float32).astype(np.float64)
    dt = torch.float32 if kind == "f32" else torch.float64
    x = torch.from_numpy(xs).to("cuda", dt)
    y = torch.full_like(x, float("nan"))
    M.apply(L, x, y, ieee=kind == "f64_ieee")
    torch.cuda.synchronize()
    ref = y.double().cpu().numpy()
    got = _partitioned(coarse, L, world, xs, kind)
    assert np.all(np.isfinite(got))
    assert np.array_equal(got, ref)
    M.close()


def test_apply_partial_copies_sum_to_the_apply(cuda):
    """hyteg_apply_partial on the whole mesh: summing the copies of every
    interface DoF in ascending macro order gives hyteg_apply's values; inside
    the macros the two agree slot by slot."""
    import torch
    import ctypes
    H = _lib()
    from paper_2305_15116_gb300 import _capi as C
    coarse = unit_square_mesh(3, 0.15, 2)
    L = 5
    M = H.Mesh(coarse.coords, coarse.cells, H.BC_NONE).refine(L)
    smap = M.dof_map(L)
    x = torch.from_numpy(random_vector(smap.max() + 1, 3)[smap]).cuda()
    y = torch.empty_like(x)
    yp = torch.full_like(x, float("nan"))
    M.apply(L, x, y, ieee=True)
    C.check(C.lib.hyteg_apply_partial(M._h, L, C.F64_IEEE, ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(yp.data_ptr()), None), "hyteg_apply_partial")
    torch.cuda.synchronize()
    ys, ps = y.cpu().numpy(), yp.cpu().numpy()
    assert np.all(np.isfinite(ps))
    order = np.argsort(smap, kind="stable")
    sums = np.zeros(smap.max() + 1)
    for s in order:  # ascending slot = ascending macro
        sums[smap[s]] = sums[smap[s]] + ps[s]
    assert np.array_equal(sums[smap], ys)
    M.close()
