"""Shared helpers of the parity tests: run the library's apply and the oracle
on the same seeded inputs and compare element by element.

Tolerances (reading of "relative" for this operator): norm-wise
||y_gpu - y_oracle||_inf <= tol_norm * ||y_oracle||_inf, plus a per-row bound
|y_gpu - y_oracle|_i <= tol_row * sum_j |a_ij x_j| (interior rows sum to zero,
so single entries can be far below the norm).
"""
from __future__ import annotations

import numpy as np

import oracle
from inputs import random_vector

# (norm-wise, per-row) tolerances per arithmetic
TOL = {
    "f64": (1e-12, 1e-13),       # float64 data, float-float arithmetic
    "f64_ieee": (1e-12, 1e-14),  # float64 data, native fp64 FMA
    "f32": (1e-6, 2e-6),         # float32 data and weights
}


def dtype_args(kind):
    import torch
    if kind == "f32":
        return torch.float32, False
    return torch.float64, kind == "f64_ieee"


def oracle_reference(coarse, level, bc=True, x_seed=1, kind="f64"):
    """Oracle matrix, x (global numbering), y and sum_j |a_ij x_j|."""
    rm = oracle.RefinedMesh(coarse.coords, coarse.cells, level, dirichlet=bc)
    A = oracle.operator_matrix(rm)
    x = random_vector(rm.n_global, x_seed)
    if kind == "f32":
        x = x.astype(np.float32).astype(np.float64)  # the fp32 apply sees fp32-rounded inputs
    y = oracle.spmv(A, x)
    absrow = abs(A) @ np.abs(x)
    return rm, x, y, absrow


def check_close(y_gpu, y_ref, absrow, kind, where=""):
    tn, tr = TOL[kind]
    assert np.all(np.isfinite(y_gpu)), f"{where}: non-finite output (unwritten slot?)"
    d = np.abs(y_gpu - y_ref)
    norm = np.abs(y_ref).max()
    assert d.max() <= tn * norm, f"{where}: norm-wise error {d.max() / norm:.3e} > {tn}"
    bad = d > tr * absrow + 1e-300
    assert not bad.any(), (f"{where}: per-row bound broken at {np.nonzero(bad)[0][:5]}: "
                           f"{d[bad][:5]} vs {(tr * absrow)[bad][:5]}")


def gpu_apply(mesh_lib, level, x_slots, kind, stream=None):
    import torch
    dt, ieee = dtype_args(kind)
    xs = torch.from_numpy(x_slots).to("cuda", dt)
    ys = torch.full_like(xs, float("nan"))
    mesh_lib.apply(level, xs, ys, ieee=ieee, stream=stream)
    torch.cuda.synchronize()
    return ys.double().cpu().numpy()
