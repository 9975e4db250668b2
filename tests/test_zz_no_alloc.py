"""hyteg_apply_host_static — the host-buffer apply that allocates nothing.

It is meant for callers that cannot let the library call cudaMalloc (a stream
being captured into a CUDA graph, real-time loops that forbid allocation after
start-up, processes whose device memory belongs to another allocator).  Its
staging lives in a fixed device array shared by all calls, so this test makes
two calls in a row with different inputs and checks each result against the
allocating entry point, hyteg_apply_host, within the parity tolerances.  It
sits in a file that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

from inputs import unit_square_mesh, unit_cube_kuhn_mesh, random_vector
from parity import TOL

pytestmark = pytest.mark.gpu


def _static_apply(H, C, M, level, code, xh, yh):
    import torch
    s = torch.cuda.current_stream().cuda_stream
    return C.lib.hyteg_apply_host_static(M._h, level, code, ctypes.c_void_p(xh.data_ptr()),
                                         ctypes.c_void_p(yh.data_ptr()), ctypes.c_void_p(s))


def _check(y_static, y_ref, kind):
    tn, _ = TOL[kind]
    assert np.all(np.isfinite(y_static))
    err = np.abs(y_static - y_ref).max()
    assert err <= tn * np.abs(y_ref).max(), err


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
    for call, seed in enumerate((11, 12)):  # two calls in a row, different inputs
        xh = torch.from_numpy(random_vector(ng, seed)[smap]).to(dt).pin_memory()
        y_ref = torch.empty_like(xh).pin_memory()
        M.apply_host(level, xh, y_ref)
        y_st = torch.full_like(xh, float("nan")).pin_memory()
        rc = _static_apply(H, C, M, level, code, xh, y_st)
        assert rc == 0, C.lib.hyteg_last_error().decode()
        _check(y_st.double().numpy(), y_ref.double().numpy(), kind)
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
