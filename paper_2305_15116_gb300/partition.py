"""The operator apply over macros partitioned across processes.

The paper's weak scaling assigns macro-primitives to processes (Sec. 6: one
macro per process); an apply then needs one exchange, of the partial rows at
the DoFs that macros of different processes share.  Here every process (rank)
owns a contiguous block of the coarse cells, refines a mesh of its own cells,
and computes y = A x with

1. hyteg_apply_partial on its mesh: complete rows inside its macros, and at
   every copy of an interface DoF (macro vertex, edge, 3D face) the partial
   row of that copy's macro;
2. an exchange of those partials with the ranks that hold other copies of the
   same DoFs (point to point, the shared copies only);
3. the sum of all copies' partials of every interface DoF in ascending global
   macro order, from zero — the order of the single-process apply, so the
   result is bitwise hyteg_apply's on the whole mesh for the float64 types —
   written to every local copy; Dirichlet DoFs get y = x.

The exchange plan (which copies go to which rank, and where each lands in the
ordered sums) is built once on the host from the global slot layout
(hyteg_dof_map of the whole mesh, no refinement needed).  Steps 2 and 3 are
tensor operations on the device of y (gather, send/recv, masked sums,
scatter); the communicator is torch.distributed by default, or any object
with the same send/recv methods.
"""
from __future__ import annotations

import numpy as np

from .mesh import Mesh, BC_NONE, BC_DIRICHLET, F64, F32, F64_IEEE
from . import _capi as C


def cell_blocks(n_cells: int, world: int) -> list[tuple[int, int]]:
    """Contiguous blocks of cells per rank, sizes differing by at most one."""
    base, extra = divmod(n_cells, world)
    out, c = [], 0
    for r in range(world):
        k = base + (1 if r < extra else 0)
        out.append((c, c + k))
        c += k
    return out


class _TorchComm:
    """Point-to-point exchange over torch.distributed (tensors on the device
    of the process group's backend: host copies for gloo)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.host = dist.get_backend(group) == "gloo"

    def exchange(self, sends: dict, recvs: dict) -> None:
        """sends: {rank: tensor}, recvs: {rank: tensor to fill}."""
        reqs, back = [], []
        for peer, t in sends.items():
            reqs.append(self.dist.isend(t.cpu() if self.host else t.contiguous(), peer, group=self.group))
        for peer, t in recvs.items():
            buf = t.new_empty(t.shape, device="cpu") if self.host else t
            reqs.append(self.dist.irecv(buf, peer, group=self.group))
            back.append((t, buf))
        for q in reqs:
            q.wait()
        for t, buf in back:
            if buf is not t:
                t.copy_(buf)


class PartitionPlan:
    """Host-side plan of one rank: its cells, what it sends to and receives
    from every other rank, and for every interface DoF it holds a copy of the
    ordered list of all copies' partials."""

    def __init__(self, coords, cells, level: int, rank: int, world: int, bc: int = BC_DIRICHLET):
        coords = np.ascontiguousarray(coords, dtype=np.float64)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        if world > 63:
            raise ValueError("at most 63 ranks")
        if not 0 <= rank < world:
            raise ValueError("rank must lie in 0 .. world - 1")
        if world > cells.shape[0]:
            raise ValueError("more ranks than coarse cells: every rank needs a macro")
        self.level, self.rank, self.world = level, rank, world
        self.blocks = cell_blocks(cells.shape[0], world)
        c0, c1 = self.blocks[rank]
        g = Mesh(coords, cells, bc)  # host-only queries of the whole mesh
        ns, _ = g.num_slots(level)
        S = ns // cells.shape[0]
        self.S = S  # slots per macro
        gid = g.dof_map(level)
        dmask = g.dirichlet_mask(level).astype(bool)
        g.close()
        lo, hi = c0 * S, c1 * S
        owner = np.repeat(np.arange(world), [(b1 - b0) * S for b0, b1 in self.blocks])
        # DoF groups: copies in ascending global slot (= ascending macro) order
        order = np.argsort(gid, kind="stable")
        gs = gid[order]
        starts = np.flatnonzero(np.r_[True, gs[1:] != gs[:-1]])
        counts = np.diff(np.r_[starts, gs.size])
        grp_of = np.empty(gs.size, dtype=np.int64)
        grp_of[order] = np.repeat(np.arange(starts.size), counts)
        # ranks holding a copy of each DoF, as a bit mask
        bits = np.left_shift(np.int64(1), owner[order].astype(np.int64))
        rmask = np.bitwise_or.reduceat(bits, starts)
        dir_grp = dmask[order[starts]]
        # the interface DoFs of this rank (several copies or Dirichlet) and
        # their copies' partials: own copies, then each peer's, by global slot
        iface_grp = (counts > 1) & ~dir_grp
        exch = iface_grp[grp_of]                                   # global slots whose partial matters
        mine = (rmask[grp_of] >> rank) & 1 == 1
        own_slots = np.flatnonzero(exch & (owner == rank))         # ascending
        self.send_slots, self.recv_slots = {}, {}
        for peer in range(world):
            if peer == rank:
                continue
            peer_has = (rmask[grp_of] >> peer) & 1 == 1
            snd = np.flatnonzero(exch & (owner == rank) & peer_has)
            rcv = np.flatnonzero(exch & (owner == peer) & mine)
            if snd.size:
                self.send_slots[peer] = snd - lo
            if rcv.size:
                self.recv_slots[peer] = rcv
        # V = [own copies' partials, the peers' in rank order]; positions of every copy
        pos_of = np.full(gs.size, -1, dtype=np.int64)
        pos_of[own_slots] = np.arange(own_slots.size)
        pos = own_slots.size
        for peer in sorted(self.recv_slots):
            r_ = self.recv_slots[peer]
            pos_of[r_] = pos + np.arange(r_.size)
            pos += r_.size
        self.n_v = pos
        self.gather_own = own_slots - lo
        my_grp = np.unique(grp_of[lo:hi][iface_grp[grp_of[lo:hi]]])
        self.max_copies = int(counts[my_grp].max()) if my_grp.size else 1
        idx = np.full((my_grp.size, self.max_copies), -1, dtype=np.int64)
        for j in range(self.max_copies):
            has = counts[my_grp] > j
            idx[has, j] = pos_of[order[starts[my_grp[has]] + j]]
        assert np.all(idx[idx != -1] >= 0)
        self.index = idx
        # write every local copy of these DoFs; Dirichlet DoFs: y = x at the copy
        loc = np.arange(lo, hi)
        lg = grp_of[loc]
        sel = iface_grp[lg]
        self.write_slots = loc[sel] - lo
        self.write_dof = np.searchsorted(my_grp, lg[sel])
        dsel = dir_grp[lg]
        self.dirichlet_slots = loc[dsel] - lo
        # the rank's own mesh: its cells over the vertices they use, renumbered
        # in ascending order (relative vertex order, and so every macro's
        # orientation and slot layout, is that of the whole mesh)
        used = np.unique(cells[c0:c1])
        self.local_cells = np.searchsorted(used, cells[c0:c1])
        self.coords = coords[used]


class PartitionedApply:
    """y = A x for this rank's block of macros (vectors in the slot layout of
    the rank's own cells), completed across ranks; see the module docstring."""

    def __init__(self, coords, cells, level: int, rank: int, world: int, bc: int = BC_DIRICHLET,
                 comm=None, partial_apply=None):
        self.plan = PartitionPlan(coords, cells, level, rank, world, bc)
        self.level = level
        self.comm = comm
        self._partial = partial_apply
        self.mesh = None
        if partial_apply is None:
            self.mesh = Mesh(self.plan.coords, self.plan.local_cells, BC_NONE).refine(level)
        self._dev = {}

    def _tables(self, device):
        import torch
        if device not in self._dev:
            p = self.plan
            t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
            self._dev[device] = dict(
                own=t(p.gather_own), index=t(np.maximum(p.index, 0)), has=t(p.index >= 0),
                send={k: t(v) for k, v in p.send_slots.items()},
                write=t(p.write_slots), wdof=t(p.write_dof), dir=t(p.dirichlet_slots))
        return self._dev[device]

    def begin(self, x, y, ieee: bool = False, stream=None) -> dict:
        """Step 1: the partial apply into y; returns the partials to send,
        {peer rank: tensor}."""
        import torch
        if self._partial is not None:
            self._partial(x, y)
        else:
            import ctypes
            from .mesh import _stream_ptr
            code = F32 if x.dtype == torch.float32 else (F64_IEEE if ieee else F64)
            C.check(C.lib.hyteg_apply_partial(self.mesh._h, self.level, code, ctypes.c_void_p(x.data_ptr()),
                                              ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))),
                    "hyteg_apply_partial")
        T = self._tables(y.device)
        return {peer: y[idx] for peer, idx in T["send"].items()}

    def receive_buffers(self, y) -> dict:
        """Empty receive buffers, {peer rank: tensor}, for step 2."""
        import torch
        return {peer: torch.empty(self.plan.recv_slots[peer].size, dtype=y.dtype, device=y.device)
                for peer in sorted(self.plan.recv_slots)}

    def complete(self, x, y, recvs: dict):
        """Step 3: the ordered sums of every interface DoF from the own and the
        received partials, written to every local copy; Dirichlet rows."""
        import torch
        p = self.plan
        T = self._tables(y.device)
        parts = [y[T["own"]]] + [recvs[peer] for peer in sorted(p.recv_slots)]
        v = torch.cat(parts) if parts else y.new_empty(0)
        # ordered sums from zero, one copy after another (absent copies add +0)
        acc = torch.zeros(p.index.shape[0], dtype=y.dtype, device=y.device)
        zero = torch.zeros((), dtype=y.dtype, device=y.device)
        for j in range(p.index.shape[1]):
            acc = acc + torch.where(T["has"][:, j], v[T["index"][:, j]], zero)
        y[T["write"]] = acc[T["wdof"]]
        y[T["dir"]] = x[T["dir"]]  # Dirichlet rows
        return y

    def apply(self, x, y, ieee: bool = False, stream=None):
        """y = A x on this rank's cells (device tensors in their slot layout);
        every rank of the partition calls it, with its own block."""
        sends = self.begin(x, y, ieee, stream)
        recvs = self.receive_buffers(y)
        if sends or recvs:
            comm = self.comm if self.comm is not None else _TorchComm()
            comm.exchange(sends, recvs)
        return self.complete(x, y, recvs)

    def close(self):
        if self.mesh is not None:
            self.mesh.close()
            self.mesh = None
