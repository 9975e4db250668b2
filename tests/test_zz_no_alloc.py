"""hyteg_apply_host_static — the host-buffer apply that allocates nothing.

It is meant for callers that cannot let the library call cudaMalloc
(real-time loops that forbid allocation after start-up, processes whose
device memory belongs to another allocator).  Its staging lives in a fixed
device array shared by all calls, so this test makes two calls in a row with
different inputs and checks that each result is bitwise the result of the
allocating entry point, hyteg_apply_host (both run the same kernels), and
that the free device memory does not drop over the two calls.  A stream under
CUDA graph capture is refused, since the call synchronises its stream.  It
sits in a file that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

from inputs import unit_square_mesh, unit_cube_kuhn_mesh, random_vector

pytestmark = pytest.mark.gpu


def _static_apply(H, C, M, level, code, xh, yh):
    import torch
    s = torch.cuda.current_stream().cuda_stream
    return C.lib.hyteg_apply_host_static(M._h, level, code, ctypes.c_void_p(xh.data_ptr()),
                                         ctypes.c_void_p(yh.data_ptr()), ctypes.c_void_p(s))


@pytest.mark.parametrize("dim,level,kind", [(2, 7, "f64"), (2, 8, "f32"), (3, 4, "f64"), (3, 4, "f32")])
def test_static_matches_allocating_apply_two_calls(cuda, dim, level, kind):
    import torch
    import paper_2305_15116_gb300 as H
    from paper_2305_15116_gb300 import _capi as C
    coarse = unit_square_mesh(4, 0.15, 0) if dim == 2 else unit_cube_kuhn_mesh(2, 0.1, 0)
    M = H.Mesh(coarse.coords, coarse.cells).refine(level)
    ns, ng = M.num_slots(level)
    smap = M.dof_map(level)
    dt = torch.float32 if kind == "f32" else torch.float64
    code = C.F32 if kind == "f32" else C.F64
    xs, refs = [], []
    for seed in (11, 12):  # reference results from the allocating entry point
        xh = torch.from_numpy(random_vector(ng, seed)[smap]).to(dt).pin_memory()
        y_ref = torch.empty_like(xh).pin_memory()
        M.apply_host(level, xh, y_ref)
        xs.append(xh)
        refs.append(y_ref)
    ys = [torch.full_like(x, float("nan")).pin_memory() for x in xs]
    # a first call commits the static array on this device (it is committed
    # when the library's device code is loaded, at the latest by the first
    # call); from then on the calls take no device memory
    warm = torch.empty_like(xs[0]).pin_memory()
    assert _static_apply(H, C, M, level, code, xs[0], warm) == 0, C.lib.hyteg_last_error().decode()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for xh, y_st in zip(xs, ys):  # two calls in a row, different inputs
        rc = _static_apply(H, C, M, level, code, xh, y_st)
        assert rc == 0, C.lib.hyteg_last_error().decode()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0, f"free device memory dropped by {free0 - free1} bytes"
    for y_st, y_ref in zip(ys, refs):
        assert np.all(np.isfinite(y_st.double().numpy()))
        assert torch.equal(y_st, y_ref)
    M.close()


def test_static_refuses_a_capturing_stream(cuda):
    """The call synchronises its stream, so under graph capture it must refuse
    (HYTEG_ESTATE) before enqueueing anything; the capture stays valid."""
    import torch
    import paper_2305_15116_gb300 as H
    from paper_2305_15116_gb300 import _capi as C
    coarse = unit_square_mesh(2, 0.15, 0)
    level = 5
    M = H.Mesh(coarse.coords, coarse.cells).refine(level)
    ns, _ = M.num_slots(level)
    xh = torch.ones(ns, dtype=torch.float64).pin_memory()
    yh = torch.zeros(ns, dtype=torch.float64).pin_memory()
    assert _static_apply(H, C, M, level, C.F64, xh, yh) == 0  # address lookup before the capture
    side = torch.cuda.Stream()
    st = ctypes.c_void_p(side.cuda_stream)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        g.capture_begin()
        try:
            rc = C.lib.hyteg_apply_host_static(M._h, level, C.F64, ctypes.c_void_p(xh.data_ptr()),
                                               ctypes.c_void_p(yh.data_ptr()), st)
            msg = C.lib.hyteg_last_error().decode()
            assert torch.cuda.is_current_stream_capturing(), "the capture was invalidated"
            torch.zeros(1, device="cuda").add_(1.0)  # keep the captured graph non-empty
        finally:
            g.capture_end()
    assert rc == C.ESTATE, (rc, msg)
    assert "captured" in msg
    torch.cuda.synchronize()
    M.close()


def test_static_rejects_vectors_above_the_limit(cuda):
    import torch
    import paper_2305_15116_gb300 as H
    from paper_2305_15116_gb300 import _capi as C
    coarse = unit_square_mesh(4, 0.15, 0)
    level = 9  # 32 x 131,841 slots x 8 B = 33.7 MB > 16 MiB
    M = H.Mesh(coarse.coords, coarse.cells).refine(level)
    ns, _ = M.num_slots(level)
    xh = torch.zeros(ns, dtype=torch.float64)
    yh = torch.zeros(ns, dtype=torch.float64)
    rc = _static_apply(H, C, M, level, C.F64, xh, yh)
    assert rc == C.EINVAL
    assert "static staging limit" in C.lib.hyteg_last_error().decode()
    M.close()
