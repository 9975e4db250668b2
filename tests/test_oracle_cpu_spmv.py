"""The oracle's multithreaded CSR loop (the CPU baseline on all host cores)
computes the same product as the oracle's scipy SpMV and as a dense product."""
import numpy as np
import pytest

import oracle
from oracle import cpu_spmv
from inputs import unit_square_mesh, unit_cube_kuhn_mesh, random_vector


@pytest.fixture(scope="module")
def built():
    cpu_spmv.build()


@pytest.mark.parametrize("dim", [2, 3])
def test_threaded_loop_equals_scipy_product(built, dim):
    coarse = unit_square_mesh(3, 0.15, 1) if dim == 2 else unit_cube_kuhn_mesh(1, 0.1, 1)
    L = 5 if dim == 2 else 3
    rm = oracle.RefinedMesh(coarse.coords, coarse.cells, L)
    A = oracle.operator_matrix(rm)
    x = random_vector(rm.n_global, 4)
    ref = oracle.spmv(A, x)
    ops = cpu_spmv.CsrOperands(A)
    for threads in (1, 2, 3, 7):
        y = cpu_spmv.spmv_threads(ops, x, threads)
        # rows in stored order, every product rounded before its add: the
        # same operations as the scalar library loop, row by row
        assert np.array_equal(y, ref), threads


def test_threaded_loop_equals_dense_product_on_a_tiny_matrix(built):
    rng = np.random.default_rng(3)
    import scipy.sparse as sp
    D = rng.standard_normal((9, 9)) * (rng.random((9, 9)) < 0.4)
    D[4, :] = 0.0  # an empty row
    x = rng.standard_normal(9)
    y = cpu_spmv.spmv_threads(cpu_spmv.CsrOperands(sp.csr_matrix(D)), x, 4)
    assert np.allclose(y, D @ x, rtol=1e-15, atol=1e-15)
    assert y[4] == 0.0


def test_host_cores_is_positive():
    assert cpu_spmv.host_cores() >= 1
