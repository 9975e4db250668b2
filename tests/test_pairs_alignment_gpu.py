"""fp32 vectors at odd element offsets (4-byte aligned views into larger
buffers): the 2D fp32 apply and sweeps copy and store a lane's two columns as
one 8-byte pair only on the rows where every vector involved is 8-byte
aligned, and element by element elsewhere.  The results must not depend on
the vectors' alignment: bitwise the same as with aligned vectors (needs a
GPU)."""
import pytest

from inputs import unit_square_mesh, random_vector

pytestmark = pytest.mark.gpu

OFFSETS = [(1, 0), (0, 1), (1, 1)]


def _views(ns, off, dtype, fill=0.0):
    import torch
    buf = torch.full((ns + 2,), fill, dtype=dtype, device="cuda")
    return buf[off:off + ns]


@pytest.mark.parametrize("L", [6, 9])
def test_fp32_apply_at_odd_offsets(cuda, L):
    import torch
    import paper_2305_15116_gb300 as H
    coarse = unit_square_mesh(4, 0.15, 0)
    M = H.Mesh(coarse.coords, coarse.cells).refine(L)
    ns, ng = M.num_slots(L)
    x = torch.from_numpy(random_vector(ng, 3)[M.dof_map(L)]).float().cuda()
    ref = M.apply(L, x, torch.empty_like(x))
    for ox, oy in OFFSETS:
        xv = _views(ns, ox, torch.float32)
        xv.copy_(x)
        yv = _views(ns, oy, torch.float32, float("nan"))
        assert xv.data_ptr() % 8 == 4 * ox and yv.data_ptr() % 8 == 4 * oy
        M.apply(L, xv, yv)
        torch.cuda.synchronize()
        assert torch.equal(yv, ref), (ox, oy)
    M.close()


def test_fp32_vcycle_at_odd_offsets(cuda):
    """Two fp32 V-cycles with b and u at odd offsets (the top level's sweeps
    read u and b and alternate between u and the level's own aligned spare
    vector) against the same cycles on aligned vectors."""
    import torch
    import paper_2305_15116_gb300 as H
    L = 7
    coarse = unit_square_mesh(4, 0.15, 0)
    M = H.Mesh(coarse.coords, coarse.cells).refine(L).solver_setup(L)
    ns, ng = M.num_slots(L)
    b = torch.from_numpy(random_vector(ng, 4)[M.dof_map(L)]).float().cuda()
    u = torch.zeros_like(b)
    for _ in range(2):
        M.vcycle(L, b, u)
    for ob, ou in OFFSETS:
        bv = _views(ns, ob, torch.float32)
        bv.copy_(b)
        uv = _views(ns, ou, torch.float32)
        for _ in range(2):
            M.vcycle(L, bv, uv)
        torch.cuda.synchronize()
        assert torch.equal(uv, u), (ob, ou)
    M.close()
