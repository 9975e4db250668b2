"""Python view of the solve server (marshalling only; include/hyteg.h)."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _capi as C
from ._capi import SOLVE_MIXED, EAGAIN, ETIMEDOUT, REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED, HytegError


@dataclass
class Result:
    status: int
    error: int
    iters: int
    cache_hit: bool
    relres: float
    queue_s: float
    run_s: float
    n_global: int
    setup_s: float = 0.0
    message: str = ""
    group: int = 1  # requests solved together in one group solve

    @property
    def finished(self) -> bool:
        return self.status in (REQ_DONE, REQ_FAILED)


def _result(r: C.Result) -> Result:
    msg = C.lib.hyteg_last_error().decode(errors="replace") if r.status == REQ_FAILED else ""
    return Result(r.status, r.error, r.iters, bool(r.cache_hit), r.relres, r.queue_s, r.run_s, r.n_global,
                  r.setup_s, msg, r.group)


class Server:
    """Poisson solve server on one GPU: `mem_cap` bytes of device arena and
    `n_workers` worker threads with one CUDA stream each."""

    def __init__(self, mem_cap: int, n_workers: int = 4, device: int = 0):
        h = ctypes.c_void_p()
        C.check(C.lib.hyteg_server_create(device, int(mem_cap), n_workers, ctypes.byref(h)), "hyteg_server_create")
        self._h = h
        self._keep = {}  # ticket -> host arrays the library writes into or reads at submit

    def submit(self, coords, cells, level: int, seed: int, noise: float = 0.1, mode: int = SOLVE_MIXED,
               rtol: float = 1e-8, max_iter: int = 100, u_out: np.ndarray | None = None,
               b_out: np.ndarray | None = None, u_lo_out: np.ndarray | None = None):
        """Enqueue one request; returns its ticket, or None when the memory cap
        refuses it for now (HYTEG_EAGAIN)."""
        coords = np.ascontiguousarray(coords, dtype=np.float64)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        for a in (u_out, b_out, u_lo_out):
            if a is not None and (a.dtype != np.float64 or not a.flags.c_contiguous):
                raise ValueError("u_out / b_out / u_lo_out must be C-contiguous float64 arrays")
        req = C.Request(int(coords.shape[1]), coords.shape[0], coords.ctypes.data_as(C.c_dblp), cells.shape[0],
                        cells.ctypes.data_as(C.c_i64p), level, mode, rtol, max_iter, seed, noise,
                        u_out.ctypes.data_as(C.c_dblp) if u_out is not None else None,
                        b_out.ctypes.data_as(C.c_dblp) if b_out is not None else None,
                        u_lo_out.ctypes.data_as(C.c_dblp) if u_lo_out is not None else None)
        t = ctypes.c_uint64()
        code = C.lib.hyteg_server_submit(self._h, ctypes.byref(req), ctypes.byref(t))
        if code == EAGAIN:
            return None
        C.check(code, "hyteg_server_submit")
        self._keep[t.value] = (u_out, b_out, u_lo_out)
        return t.value

    def poll(self, ticket: int) -> Result:
        r = C.Result()
        C.check(C.lib.hyteg_server_poll(self._h, ticket, ctypes.byref(r)), "hyteg_server_poll")
        return _result(r)

    def wait(self, ticket: int, timeout: float = 600.0) -> Result | None:
        """The finished request's result, or None if the timeout ran out."""
        r = C.Result()
        code = C.lib.hyteg_server_wait(self._h, ticket, timeout, ctypes.byref(r))
        if code == ETIMEDOUT:
            return None
        C.check(code, "hyteg_server_wait")
        return _result(r)

    def release(self, ticket: int) -> None:
        C.check(C.lib.hyteg_server_release(self._h, ticket), "hyteg_server_release")
        self._keep.pop(ticket, None)

    def inject_alloc_failures(self, count: int) -> None:
        """The next `count` arena allocations fail (host-side fault injection)."""
        C.check(C.lib.hyteg_server_inject_alloc_failures(self._h, count), "hyteg_server_inject_alloc_failures")

    def stats(self) -> dict:
        s = C.ServerStats()
        C.check(C.lib.hyteg_server_stats_get(self._h, ctypes.byref(s)), "hyteg_server_stats_get")
        return {k: getattr(s, k) for k, _ in C.ServerStats._fields_}

    def close(self) -> None:
        if getattr(self, "_h", None):
            C.lib.hyteg_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
