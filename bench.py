#!/usr/bin/env python3
"""Throughput of the matrix-free P1 operator apply y = A x on GB300.

One step = one apply on the 2D workload "square32jit_L11": the unit square as
4x4 cells x 2 triangles = 32 jittered macro-triangles, refined to level 11
(67,125,249 distinct DoFs, 67,207,200 slots), float64 vectors, x ~ U[-1,1].
The metric is distinct DoF updates per second (GDoF/s) — the paper's
throughput unit (Sec. 5.2 reports GFLOP/s of the same kernel at 13 flop per
update).  Inputs (0.54 GB x + 0.54 GB y) are larger than the 129 MB L2, so
the L2 is not flushed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent replica of the
workload on its own GPU (the apply has no data-path collective at this size);
`value` sums all ranks' DoF updates over the slowest rank's time.
Prints ONE JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GDoF-updates/s of A*x (P1 stiffness apply, distinct DoFs)"
UNIT = "GDoF/s"
WORKLOAD = "square32jit_L11"
FP64_PEAK_GOPS = 625.0  # nominal GB300 dense fp64: 1.25 TFLOP/s, an FMA counting two
CPU_SAMPLE_LEVEL = 10  # the oracle's sample of the 2D workload (assembly takes about a minute)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000,
                   help="timed applies (default 2000: about 0.5 s, so that the clock sampler sees ~10 samples)")
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-variants", action="store_true", help="skip the fp32 / 3D / native-fp64 lines")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--workload", default=WORKLOAD, help="workload to time (default: the 2D level-11 case)")
    p.add_argument("--dtype", default="f64", choices=["f64", "f32", "f64_ieee"])
    p.add_argument("--level", type=int, default=None,
                   help="override the refinement level (smaller cases for ncu captures; not a bench line)")
    p.add_argument("--serve-requests", type=int, default=4096,
                   help="requests of the solve-server workload timed after the apply (0: skip)")
    p.add_argument("--serve-workers", type=int, default=8)
    p.add_argument("--profile", action="store_true",
                   help="only run warm-up + timed applies (for profilers): no e2e, variants or CPU baseline")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_config(name):
    from inputs import WORKLOADS
    w = WORKLOADS[name]
    return w


def describe(name, n_global, n_slots):
    from inputs import WORKLOADS
    w = WORKLOADS[name]
    if w["dim"] == 2:
        shape = f"unit square, {w['k']}x{w['k']} cells x 2 triangles = {2 * w['k'] ** 2} macro-triangles"
    else:
        shape = f"unit cube, {w['k']}^3 cells x 6 Kuhn tets = {6 * w['k'] ** 3} macro-tets"
    jit = f", interior coarse vertices jittered U[-{w['jitter']}h, {w['jitter']}h] (seed {w['mesh_seed']})" \
        if w["jitter"] else ""
    disc = "P2 (vertex + edge DoF)" if w.get("op") == "p2" else "P1"
    return (f"{name}: {w['dim']}D {disc} Laplacian apply, {shape}{jit}, level {w['level']}, "
            f"{n_global} DoFs ({n_slots} slots), x ~ U[-1,1] seed {w['x_seed']}, Dirichlet rows identity")


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons, with timestamps."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--id={index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(", ") for r in self.f.read().strip().splitlines() if r.strip()]
        self.f.close()
        os.unlink(self.f.name)
        return rows

    @staticmethod
    def summarise(rows, t0, t1):
        import datetime as dt
        sel, allr = [], []
        for r in rows:
            if len(r) < 9:
                continue
            try:
                ts = dt.datetime.strptime(r[0].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                continue
            allr.append((ts, r))
            if t0 - 0.05 <= ts <= t1 + 0.05:
                sel.append(r)
        note = None
        if not sel and allr:  # timed window shorter than the sampling period
            mid = 0.5 * (t0 + t1)
            sel = [min(allr, key=lambda a: abs(a[0] - mid))[1]]
            note = "timed region shorter than the 50 ms sampling period; nearest sample"
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in sel if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in sel if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in sel for i in range(4) if r[5 + i].strip() == "Active"})
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
               "reasons": reasons, "samples": len(sel)}
        if note:
            out["note"] = note
        return out


# ---------------------------------------------------------------- setup
def setup(name, device, dtype_code, level=None):
    import torch
    import paper_2305_15116_gb300 as H
    from inputs import workload, random_vector
    from inputs import WORKLOADS
    coarse, L, seed = workload(name, level)
    p2 = WORKLOADS[name].get("op") == "p2"
    M = H.Mesh(coarse.coords, coarse.cells).refine(L)
    ns, ng = M.p2_num_slots(L) if p2 else M.num_slots(L)
    smap = M.p2_dof_map(L) if p2 else M.dof_map(L)
    x = random_vector(ng, seed)
    tdt = torch.float32 if dtype_code == H.F32 else torch.float64
    xs = torch.from_numpy(x[smap]).to(device=device, dtype=tdt)
    ys = torch.empty_like(xs)
    n = 1 << L
    interior = coarse.n_cells * ((n - 1) * (n - 2) // 2 if coarse.dim == 2 else (n - 1) * (n - 2) * (n - 3) // 6)
    slab = True  # every apply kernel writes every slot (interface copies included)
    # the library's kernel launches per apply: 2D one (macro interiors and
    # interface points together); 3D the slab kernel (or the row kernel and
    # its row-end companion) and the interface reduction; P2 the row and
    # boundary kernels and the vertex and edge reductions
    if p2:
        launches = 4
    elif coarse.dim == 2:
        launches = 1
    else:
        launches = 2 if n <= 64 else 3
    if p2:
        kernel = "k_p2_apply"
        raw = lambda l, c, xp, yp, sp: M.p2_apply_timed(l, c, xp, yp, sp, 0, 0, 0)
        timed = M.p2_apply_timed
    else:
        kernel = "k_interior2d" if coarse.dim == 2 else ("k_slab3d" if n <= 64 else "k_row3d")
        raw, timed = M.apply_raw, M.apply_timed
    return dict(M=M, L=L, ns=ns, ng=ng, xs=xs, ys=ys, smap=smap, x_global=x, coarse=coarse,
                interior=interior, elem=4 if dtype_code == H.F32 else 8, code=dtype_code, launches=launches,
                slab=slab or p2, kernel=kernel, apply_raw=raw, apply_timed=timed, op="p2" if p2 else "p1")


L2_BYTES = 129 * 2 ** 20


def timed_applies(w, steps, warmup, stream, barrier=None, flush=None):
    """Warm-up, then exactly `steps` applies timed with CUDA events on the
    launching stream; per-kernel durations from events recorded by the
    library between its two launches.  With `flush` (a device buffer larger
    than L2) the buffer is overwritten before every timed apply, so that no
    apply finds its vectors in L2; the per-apply times then exclude the
    flush."""
    import torch
    M, L, code = w["M"], w["L"], w["code"]
    xp, yp, sp = w["xs"].data_ptr(), w["ys"].data_ptr(), stream.cuda_stream
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    with torch.cuda.stream(stream):
        for row in ev:  # create the events (torch creates them lazily)
            for e in row:
                e.record(stream)
        for _ in range(warmup):
            w["apply_raw"](L, code, xp, yp, sp)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # an NVTX range around the timed applies, so that a profiler can select
    # them (the refinement's autotuner launches the same kernels before)
    torch.cuda.nvtx.range_push("timed_applies")
    t0 = time.time()
    start.record(stream)
    for k in range(steps):
        if flush is not None:
            with torch.cuda.stream(stream):
                flush.fill_(k)
        w["apply_timed"](L, code, xp, yp, sp, ev[k][0].cuda_event, ev[k][1].cuda_event, ev[k][2].cuda_event)
    end.record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    torch.cuda.nvtx.range_pop()
    if barrier:
        barrier()
    total_ms = start.elapsed_time(end)
    interior_ms = [ev[k][0].elapsed_time(ev[k][1]) for k in range(steps)]
    iface_ms = [ev[k][1].elapsed_time(ev[k][2]) for k in range(steps)]
    apply_ms = [ev[k][0].elapsed_time(ev[k][2]) for k in range(steps)]
    return dict(total_ms=total_ms, interior_ms=float(np.mean(interior_ms)), iface_ms=float(np.mean(iface_ms)),
                apply_ms=float(np.mean(apply_ms)), t0=t0, t1=t1)


def graph_replay_us(w, reps, stream):
    """Mean device time of one apply when it is replayed from a CUDA graph
    (the library's apply allocates nothing and never synchronises, so it can
    be captured)."""
    import torch
    M, L, code = w["M"], w["L"], w["code"]
    xp, yp = w["xs"].data_ptr(), w["ys"].data_ptr()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        M.apply_raw(L, code, xp, yp, stream.cuda_stream)  # warm-up outside the capture
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=stream):
            M.apply_raw(L, code, xp, yp, torch.cuda.current_stream().cuda_stream)
        for _ in range(5):
            g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
    return 1e3 * e0.elapsed_time(e1) / reps


def batched_small(w, count, stream, reps=50):
    """`count` products of the small mesh (distinct vector pairs, as from as
    many requests): one hyteg_apply each against one hyteg_apply_batch for
    all of them, timed with CUDA events on the launching stream."""
    import torch
    import paper_2305_15116_gb300 as H
    M, L = w["M"], w["L"]
    g = torch.Generator(device="cpu").manual_seed(7)
    xs = [torch.rand(w["ns"], generator=g, dtype=torch.float64).to(w["xs"].device) for _ in range(count)]
    ys = [torch.empty_like(x) for x in xs]
    out = {}
    with torch.cuda.stream(stream):
        for mode in ("one launch per product", "hyteg_apply_batch"):
            def run():
                if mode == "hyteg_apply_batch":
                    H.apply_batch([M] * count, [L] * count, xs, ys, stream=stream)
                else:
                    for x, y in zip(xs, ys):
                        M.apply_raw(L, H.F64, x.data_ptr(), y.data_ptr(), stream.cuda_stream)
            for _ in range(3):
                run()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                run()
            e1.record(stream)
            torch.cuda.synchronize()
            us = 1e3 * e0.elapsed_time(e1) / reps
            out[mode] = {"us_per_batch": us, "GDoF_per_s": count * w["ng"] / (us * 1e-6) / 1e9}
    # the two agree bit for bit
    ref = [torch.empty_like(x) for x in xs]
    for x, r in zip(xs, ref):
        M.apply(L, x, r, stream=stream)
    H.apply_batch([M] * count, [L] * count, xs, ys, stream=stream)
    torch.cuda.synchronize()
    out["bitwise_equal"] = all(torch.equal(a, b) for a, b in zip(ys, ref))
    out["workload"] = f"{count} products on the 2-macro level-7 mesh (16,641 DoFs each), float64 data"
    return out


def interior_bytes(w):
    """Algorithmic bytes of one launch of the dominant kernel: every slot of
    every macro is read once and written once (the 2D apply writes its
    interface points in the same launch, the 3D and P2 kernels write the
    macro-boundary partials)."""
    return w["elem"] * (w["ns"] + (w["ns"] if w["slab"] else w["interior"]))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mp = json.load(f)
        return float(mp["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def ncu_traffic(kernel_key):
    """Per-launch DRAM bytes from the committed ncu summary, only while the
    kernel source is unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            data = json.load(f)
        entry = data[kernel_key]
    except Exception:
        return None
    src = os.path.join(ROOT, entry["source"])
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        arith = os.path.join(ROOT, "paper_2305_15116_gb300", "csrc", "arith.cuh")
        h2 = hashlib.sha256(open(arith, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    if entry.get("source_sha") != h or entry.get("arith_sha") != h2:
        return None
    return entry["dram_bytes_per_launch"]


# ---------------------------------------------------------------- solver
def vcycle_bytes(M, L, elem, nu1=3, nu2=3):
    """Algorithmic bytes of one V(nu1, nu2) cycle from level L (element size
    elem, 2D fused sweeps): per level k >= 1 with S_k slots, the pre-sweeps
    (nu1 on the finest level, nu1 - 1 below, where the restriction has done
    the first one), the residual sweep and nu2 post-sweeps each read u and b
    and write one vector (3 elem per slot); the restriction reads r (elem per
    fine slot) and writes b, and below level 1 also u, of the coarser level
    reading its inverse diagonal (3 elem per coarse slot, 1 for level 0); the
    prolongation reads the coarse correction and updates u (elem per coarse
    slot, 2 elem per fine slot); an odd number of sweeps copies u back
    (2 elem per slot).  Level 0: the direct solve reads b and writes u."""
    S = [M.num_slots(k)[0] for k in range(L + 1)]
    total = 2 * elem * S[0]
    for k in range(L, 0, -1):
        pre = nu1 if k == L else nu1 - 1
        total += 3 * elem * S[k] * (pre + 1 + nu2)
        total += elem * S[k] + (3 if k - 1 > 0 else 1) * elem * S[k - 1]
        total += elem * S[k - 1] + 2 * elem * S[k]
        if (pre + nu2) % 2:
            total += 2 * elem * S[k]
    return total


def solve_workload(device, stream, reps=3, rtol=1e-10):
    """Poisson solve -Lap u = f on the 32-macro jittered mesh at level 10,
    f = sin(pi x) sin(pi y) + 0.1 N(0,1) (noise per global DoF from seed 2),
    lumped-mass right-hand side, u = 0 on the boundary: fp32 V(3,3) cycles in
    float64 iterative refinement against plain float64 V(3,3) cycles."""
    import torch
    import paper_2305_15116_gb300 as H
    from inputs import workload, random_normal
    name = "square32jit_L10_solve"
    coarse, L, seed = workload(name)
    M = H.Mesh(coarse.coords, coarse.cells).refine(L).solver_setup(L, 3, 3, 2.0 / 3.0)
    ns, ng = M.num_slots(L)
    smap = M.dof_map(L)
    xyz = M.slot_coords(L)
    f = np.sin(np.pi * xyz[:, 0]) * np.sin(np.pi * xyz[:, 1]) + 0.1 * random_normal(ng, seed)[smap]
    b = M.lumped_mass(L) * f
    b[M.dirichlet_mask(L)] = 0.0
    bd = torch.from_numpy(b).to(device)
    u = torch.zeros_like(bd)
    ulo = torch.zeros_like(bd)
    out = {"workload": f"{name}: 2D Poisson, 32 jittered macro-triangles, level {L}, {ng} DoFs; "
                       "f = sin(pi x) sin(pi y) + 0.1 N(0,1), lumped mass, u = 0 on the boundary; "
                       f"V(3,3) weighted Jacobi (2/3), rtol {rtol}"}
    runs = (("mixed_fp32_vcycles_two_part_refinement", H.SOLVE_MIXED, True),
            ("fp64_vcycles_two_part_refinement", H.SOLVE_F64, True),
            ("mixed_fp32_vcycles_fp64_refinement", H.SOLVE_MIXED, False),
            ("fp64_vcycles", H.SOLVE_F64, False))
    for label, mode, two in runs:
        def run():
            u.zero_()
            ulo.zero_()
            if two:
                return M.solve_two_part(L, bd, u, ulo, mode=mode, rtol=rtol, max_iter=200, stream=stream)
            return M.solve(L, bd, u, mode=mode, rtol=rtol, max_iter=200, stream=stream)
        run()  # warm-up
        times, its, rels = [], [], []
        for _ in range(reps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            it, rel = run()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t)
            its.append(it)
            rels.append(rel)
        out[label] = {"solves_per_s": 1.0 / float(np.median(times)), "ms_per_solve": 1e3 * float(np.median(times)),
                      "iterations": its[-1], "relres": rels[-1], "reached_rtol": bool(rels[-1] <= rtol)}
    # one fp32 V(3,3) cycle on its own: device time and its algorithmic bytes
    b32 = bd.float()
    u32 = torch.zeros_like(b32)
    with torch.cuda.stream(stream):
        for _ in range(3):
            M.vcycle(L, b32, u32, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed_vcycles")
        e0.record(stream)
        for _ in range(20):
            M.vcycle(L, b32, u32, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    ms = e0.elapsed_time(e1) / 20
    vb = vcycle_bytes(M, L, 4)
    peak, peak_kind = measured_peaks()
    out["vcycle_fp32"] = {
        "ms": ms, "algorithmic_bytes": vb, "achieved_GBps": vb / (ms * 1e-3) / 1e9,
        "frac": vb / (ms * 1e-3) / 1e9 / peak, "peak": peak, "peak_kind": f"{peak_kind} copy bandwidth",
        "share_of_mixed_solve": ms * out["mixed_fp32_vcycles_two_part_refinement"]["iterations"]
        / out["mixed_fp32_vcycles_two_part_refinement"]["ms_per_solve"],
        "note": "one fp32 V(3,3) cycle from level 10 down to level 0 (hyteg_vcycle), 20 cycles timed with CUDA "
                "events; algorithmic bytes: every sweep reads u and b and writes its result, the residual sweep "
                "likewise, the restriction reads r and writes b and u of the coarser level, the prolongation "
                "reads the coarse correction and updates u, an odd sweep count copies u back (4 B per slot "
                "each)"}
    out["note"] = ("two_part: the iterate is u + u_lo, two float64 vectors (hyteg_solve_two_part), which reaches "
                   "rtol; the float64-iterate loops stop at rtol or when two iterations in a row each reduce "
                   "the residual by less than 10 %: at level 10 the rounding of a float64 solution leaves a "
                   "relative residual of about 1.9e-10 (pinned by the oracle's exactly rounded residual at "
                   "levels 4-6, 4x per level)")
    M.close()
    return out


def group_workload(device, stream, count=8, level=7, reps=3, rtol=1e-10):
    """`count` Poisson problems on different 2D meshes (8 to 12 jittered
    macro-triangles) at one level, solved one after another with
    hyteg_solve_two_part against all at once with hyteg_solve_two_part_group
    (one launch per solve step for all problems still iterating); the
    results agree bit for bit."""
    import torch
    import paper_2305_15116_gb300 as H
    from inputs import rect_mesh
    meshes, bs = [], []
    for k in range(count):
        c = rect_mesh(2, 2 + k % 2, 0.15, k)
        M = H.Mesh(c.coords, c.cells).refine(level).solver_setup(level)
        b = torch.empty(M.num_slots(level)[0], dtype=torch.float64, device=device)
        M.poisson_rhs(level, 100 + k, 0.1, b, stream=stream)
        meshes.append(M)
        bs.append(b)
    us = [torch.zeros_like(b) for b in bs]
    ls = [torch.zeros_like(b) for b in bs]

    def alone():
        out = []
        for M, b, u, lo in zip(meshes, bs, us, ls):
            u.zero_()
            lo.zero_()
            out.append(M.solve_two_part(level, b, u, lo, rtol=rtol, max_iter=100, stream=stream))
        return out

    def grouped():
        for u, lo in zip(us, ls):
            u.zero_()
            lo.zero_()
        return H.solve_two_part_group(meshes, level, bs, us, ls, rtol=rtol, max_iter=100, stream=stream)

    out = {"workload": f"{count} Poisson problems, 2D, 8 or 12 jittered macro-triangles each, level {level}, "
                       f"rtol {rtol}, fp32 V(3,3) cycles in two-part float64 refinement"}
    res = {}
    for label, fn in (("one_after_another", alone), ("group", grouped)):
        fn()  # warm-up (the single solves' second run replays their cycles as CUDA graphs)
        times = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            r = fn()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t)
        res[label] = ([u.clone() for u in us], r)
        out[label] = {"ms": 1e3 * min(times), "iterations": [it for it, _ in r],
                      "relres_max": max(rel for _, rel in r)}
    out["speedup"] = out["one_after_another"]["ms"] / out["group"]["ms"]
    out["bitwise_equal"] = all(torch.equal(a, b) for a, b in zip(res["one_after_another"][0], res["group"][0]))
    for M in meshes:
        M.close()
    return out


# ---------------------------------------------------------------- solve server
def serve_workload(n_requests, workers, cap_bytes=40 << 30, rtol=1e-10, mode=None, rate=2000.0):
    """The solve server under the synthetic request stream of inputs.serving:
    Poisson arrivals at 2000/s, half 2D (4..64 macro-triangles, levels 5..10),
    half 3D (6..384 macro-tets, levels 3..6), each request a lumped-mass
    right-hand side with its own noise seed, solved to rtol with fp32 V(3,3)
    cycles in float64 refinement (mode None) or float64 cycles; the solution
    of every request is copied back to host memory.  Requests refused by the
    memory cap are retried in order.  Latency runs from a request's arrival
    to the end of its work.  A solve whose residual stops falling above rtol
    (the float64 floor of 2D level 10 is about 1.8e-10) ends there; the line
    counts those apart."""
    import collections
    import paper_2305_15116_gb300 as H
    if mode is None:
        mode = H.SOLVE_MIXED
    from inputs.serving import request_stream, coarse_mesh
    reqs = request_stream(n_requests, rate=rate)
    ng_of = {}
    for q in reqs:  # DoF counts from the library's host-side layout (untimed)
        key = (q.dim, q.shape, q.level)
        if key not in ng_of:
            c = coarse_mesh(q.dim, q.shape)
            M = H.Mesh(c.coords, c.cells)
            ng_of[key] = M.num_slots(q.level)[1]
            M.close()
    pool = collections.defaultdict(list)

    def buf(n):
        return pool[n].pop() if pool[n] else np.empty(n)

    sv = H.Server(cap_bytes, workers)
    # warm-up: one small request per dimension (module load, first launches)
    for dim, shape, lev in ((2, (2, 1), 5), (3, (1, 1, 1), 3)):
        c = coarse_mesh(dim, shape)
        t = sv.submit(c.coords, c.cells, lev, 1, 0.1, rtol=rtol, mode=mode)
        sv.wait(t, 600)
        sv.release(t)
    pending = collections.deque(reqs)
    retry = collections.deque()
    outstanding = {}
    lat, run, queue_s, iters, rels, ngs, setup, missed, groups = [], [], [], [], [], [], [], [], []
    hits = failed = eagain = 0
    errors = collections.Counter()
    t0 = time.perf_counter()
    t_end = t0
    while pending or retry or outstanding:
        now = time.perf_counter() - t0
        progressed = False
        while retry or (pending and pending[0].arrival_s <= now):
            q = retry[0] if retry else pending[0]
            c = coarse_mesh(q.dim, q.shape)
            n = ng_of[(q.dim, q.shape, q.level)]
            u = buf(n)
            ts = time.perf_counter() - t0
            t = sv.submit(c.coords, c.cells, q.level, q.rhs_seed, 0.1, mode=mode, rtol=rtol, max_iter=100, u_out=u)
            if t is None:
                pool[n].append(u)
                if not retry:
                    retry.append(pending.popleft())
                eagain += 1
                break
            (retry if retry and retry[0] is q else pending).popleft()
            outstanding[t] = (q, ts, u, n)
            progressed = True
        for t in list(outstanding):
            r = sv.poll(t)
            if not r.finished:
                continue
            q, ts, u, n = outstanding.pop(t)
            sv.release(t)
            pool[n].append(u)
            progressed = True
            if r.status != H.REQ_DONE:
                failed += 1
                errors[f"{r.error}: {r.message}"] += 1
                continue
            done_at = ts + r.queue_s + r.run_s
            t_end = max(t_end, t0 + done_at)
            lat.append(done_at - q.arrival_s)
            run.append(r.run_s)
            setup.append(r.setup_s)
            queue_s.append(r.queue_s)
            iters.append(r.iters)
            rels.append(r.relres)
            groups.append(r.group)
            if r.relres > rtol:
                missed.append((q.dim, list(q.shape), q.level, r.iters, r.relres))
            ngs.append(r.n_global)
            hits += int(r.cache_hit)
        if not progressed:
            time.sleep(0.0002)
    span = t_end - t0
    st = sv.stats()
    sv.close()
    pct = lambda v, p: float(np.percentile(np.asarray(v) * 1e3, p)) if v else None
    return {
        "workload": (f"solve server, {n_requests} requests of the synthetic stream (Poisson arrivals 2000/s, seed 3; "
                     "half 2D: 4..64 jittered macro-triangles, levels 5..10; half 3D: 6..384 jittered macro-tets, "
                     f"levels 3..6; lumped-mass RHS with 0.1 N(0,1) Philox noise per request seed); rtol {rtol}, "
                     + ("fp32 V(3,3) cycles in float64 refinement" if mode == H.SOLVE_MIXED else
                        "float64 V(3,3) cycles") + "; every solution copied to host memory; "
                     f"{workers} worker streams, each solving up to 8 queued requests of one class (dimension, "
                     f"level) as one group; {cap_bytes >> 30} GiB device arena"),
        "offered_rate_per_s": rate,
        "solves_per_s": len(lat) / span, "gdofs_solved_per_s": float(np.sum(ngs)) / span / 1e9,
        "latency_ms_p50": pct(lat, 50), "latency_ms_p99": pct(lat, 99),
        "service_ms_p50": pct(run, 50), "service_ms_p99": pct(run, 99), "queue_ms_p50": pct(queue_s, 50),
        "setup_ms_p50": pct(setup, 50), "setup_share": float(np.sum(setup) / np.sum(run)) if run else None,
        "span_s": span, "done": len(lat), "failed": failed, "failures": dict(errors.most_common(5)),
        "admission_retries": eagain,
        "cache_hits": hits, "evictions": st["evictions"], "iterations_mean": float(np.mean(iters)) if iters else None,
        "relres_max": float(np.max(rels)) if rels else None,
        "reached_rtol": bool(rels and max(rels) <= rtol),
        "reached_rtol_share": float(np.mean(np.asarray(rels) <= rtol)) if rels else None,
        "not_reached_rtol": [dict(zip(("dim", "shape", "level", "iters", "relres"), m)) for m in missed[:8]],
        "group_size_mean": float(np.mean(groups)) if groups else None,
        "grouped_share": float(np.mean(np.asarray(groups) > 1)) if groups else None,
        "group_solves": st["group_solves"],
    }


# ---------------------------------------------------------------- CPU oracle
def cpu_oracle_run(steps, warmup, single_steps=3):
    """The oracle's CSR product on the host cores, on a bounded sample of the
    workload: the same 32-macro mesh at level 10 (16.8M DoFs, the largest
    level whose assembly by the oracle fits the benchmark's time), its FP64
    matrix assembled outside the timed region.  Times the oracle's plain C
    row loop (oracle/csr_spmv.c) on every host core the process may use and
    on one, and scipy's product (oracle.spmv) on one.  Returns a dict."""
    import oracle
    from oracle import cpu_spmv
    from inputs import workload, random_vector
    cpu_spmv.build()
    coarse, L, seed = workload(WORKLOAD, level=CPU_SAMPLE_LEVEL)
    rm = oracle.RefinedMesh(coarse.coords, coarse.cells, L)
    A = oracle.operator_matrix(rm)
    x = random_vector(rm.n_global, seed)
    ops = cpu_spmv.CsrOperands(A)
    cores = cpu_spmv.host_cores()
    y = np.empty(rm.n_global)

    def timed(fn, n, w):
        for _ in range(w):
            fn()
        ts = []
        for _ in range(n):
            t = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t)
        return ts

    all_ts = timed(lambda: cpu_spmv.spmv_threads(ops, x, cores, y), steps, warmup)
    one_ts = timed(lambda: cpu_spmv.spmv_threads(ops, x, 1, y), single_steps, 1)
    scipy_ts = timed(lambda: oracle.spmv(A, x), single_steps, 1)
    ng = rm.n_global
    sample = (f"{WORKLOAD} mesh at level {CPU_SAMPLE_LEVEL} ({ng} DoFs, {A.nnz} stored entries): the oracle's "
              f"assembled FP64 CSR matrix, one product y = A x per step, plain C row loop on {cores} host "
              f"threads (OpenMP, the process's affinity mask), assembly outside the timed region")
    return {"n_global": ng, "cores": cores, "all_core_s": all_ts, "one_core_s": one_ts, "scipy_one_core_s": scipy_ts,
            "sample": sample}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    steps, warmup = args.steps, max(args.warmup, 1)
    r = cpu_oracle_run(steps, warmup)
    ng, ts = r["n_global"], r["all_core_s"]
    total = sum(ts)
    value = ng * steps / total / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": steps, "warmup": warmup,
        "ms_per_step": 1e3 * total / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + f" (oracle sample at level {CPU_SAMPLE_LEVEL})",
                   "parallelism": f"{r['cores']} host threads"},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": r["cores"], "kind": "oracle", "sample": r["sample"],
                         "single_thread": ng / min(r["one_core_s"]) / 1e9,
                         "scipy_single_thread": ng / min(r["scipy_one_core_s"]) / 1e9},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- replicas
def max_over_ranks(v, device=None):
    """The largest value of v over the ranks of the default process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(local_ms, units_per_rank, world, reduce_max=None):
    """Whole-job throughput of `world` replicas that each processed
    units_per_rank units in local_ms milliseconds: the job takes the slowest
    rank's time (max over ranks), and the value is all ranks' units over it,
    in G units per second.  Returns (job ms, value)."""
    ms = reduce_max(local_ms) if (reduce_max is not None and world > 1) else float(local_ms)
    return ms, units_per_rank * world / (ms * 1e-3) / 1e9


# ---------------------------------------------------------------- main
def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    barrier = (lambda: dist.barrier(device_ids=[local])) if world > 1 else None
    import paper_2305_15116_gb300 as H

    stream = torch.cuda.Stream(device=device)
    code = {"f64": H.F64, "f32": H.F32, "f64_ieee": H.F64_IEEE}[args.dtype]
    w = setup(args.workload, device, code, args.level)
    torch.cuda.synchronize()
    if args.profile:
        r = timed_applies(w, args.steps, args.warmup, stream)
        if rank == 0:
            print(json.dumps({"profile": args.workload, "level": w["L"], "dtype": args.dtype,
                              "ms_per_step": r["total_ms"] / args.steps, "kernel_ms": r["interior_ms"],
                              "interface_ms": r["iface_ms"]}), flush=True)
        return 0

    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    time.sleep(0.2)
    r = timed_applies(w, args.steps, args.warmup, stream, barrier)
    clocks = ClockSampler.summarise(sampler.stop(), r["t0"], r["t1"]) if sampler else None

    reduce_max = (lambda v: max_over_ranks(v, device)) if world > 1 else None
    total_ms, value = job_rate(r["total_ms"], w["ng"] * args.steps, world, reduce_max)
    ms_per_step = total_ms / args.steps
    dtype_label = {"f64": "f64 data, float-float (2 x f32) arithmetic", "f32": "f32",
                   "f64_ieee": "f64 (native fp64 FMA)"}[args.dtype]

    # end to end through the C ABI with host buffers: every step copies its x
    # to the device and its y back inside the timed region; the library
    # pipelines the copies of consecutive steps with the applies
    xh = w["xs"].cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    e2e_steps = max(3, min(args.steps, 20))
    w["M"].apply_host_batch(w["L"], [xh] * 2, [yh] * 2, stream=stream)
    if barrier:
        barrier()
    t = time.perf_counter()
    w["M"].apply_host_batch(w["L"], [xh] * e2e_steps, [yh] * e2e_steps, stream=stream)
    e2e_ms, e2e_rate = job_rate(1e3 * (time.perf_counter() - t) / e2e_steps, w["ng"], world, reduce_max)
    e2e = {"value": e2e_rate, "unit": UNIT,
           "h2d_bytes_per_step": int(xh.numel() * xh.element_size()),
           "d2h_bytes_per_step": int(yh.numel() * yh.element_size())}
    del xh, yh

    peak, peak_kind = measured_peaks()
    ib = interior_bytes(w)
    achieved = ib / (r["interior_ms"] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": f"{w['kernel']} ({args.dtype})", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_kind": f"{peak_kind} copy bandwidth",
                "traffic": ncu_traffic(f"{w['kernel']}_{args.dtype}_{args.workload}"),
                "algorithmic_bytes_per_launch": ib,
                "interior_ms": r["interior_ms"], "interface_ms": r["iface_ms"]}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype_label, "data": "synthetic",
        "config": {"workload": describe(args.workload, w["ng"], w["ns"]), "dofs": w["ng"], "slots": w["ns"],
                   "l2": "inputs larger than L2 (x+y = %.2f GB per apply), no flush" % (2 * w["ns"] * 8 / 1e9),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": w["launches"] * args.steps,
        "clocks": clocks,
        "impl": "ours",
    }
    del w
    torch.cuda.empty_cache()

    if args.level is not None:
        line["config"]["note"] = f"level overridden to {args.level}: not the benchmark configuration"
    if rank == 0 and world == 1 and not args.no_variants:
        variants = []
        for name, vcode, label in ((WORKLOAD, H.F64, "f64 data, float-float arithmetic"),
                                   (WORKLOAD, H.F32, "f32"), (WORKLOAD, H.F64_IEEE, "f64 native fma"),
                                   ("cube384jit_L6", H.F64, "f64 data, float-float arithmetic"),
                                   ("cube384jit_L6", H.F32, "f32"),
                                   ("cube384jit_L6", H.F64_IEEE, "f64 native fma"),
                                   ("square32jit_P2_L10", H.F64, "f64 data, float-float arithmetic"),
                                   ("square32jit_P2_L10", H.F32, "f32"),
                                   ("square32jit_P2_L10", H.F64_IEEE, "f64 native fma")):
            if name == args.workload and vcode == code:
                continue
            v = setup(name, device, vcode)
            steps = min(args.steps, 100)
            # vectors within three times the L2 are timed with an L2 flush
            # before every apply (the value is then from the per-apply events);
            # larger ones back to back like the headline: an apply streams
            # them in the same order, so nothing survives in L2 from one
            # apply to the next, while the flush's write leaves the L2 full
            # of dirty lines whose write-back would land in the timed apply
            small = 2 * v["ns"] * v["elem"] < 3 * L2_BYTES
            flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=device) if small else None
            rv = timed_applies(v, steps, args.warmup, stream, flush=flush)
            del flush
            vb = interior_bytes(v)
            vms = rv["apply_ms"] if small else rv["total_ms"] / steps
            variants.append({
                "workload": name, "dtype": label, "kernel": v["kernel"],
                "value": v["ng"] / (vms * 1e-3) / 1e9,
                "unit": UNIT, "ms_per_step": vms,
                "l2": ("flushed before every apply (x+y = %.0f MB)" if small else
                       "inputs larger than L2 (x+y = %.0f MB), no flush") % (2 * v["ns"] * v["elem"] / 1e6),
                "interior_GBps": vb / (rv["interior_ms"] * 1e-3) / 1e9,
                "interior_frac": vb / (rv["interior_ms"] * 1e-3) / 1e9 / peak,
                "interior_ms": rv["interior_ms"], "interface_ms": rv["iface_ms"],
                "traffic": ncu_traffic("%s_%s_%s" % ("k_p2_rows" if v["op"] == "p2" else v["kernel"],
                                                     {H.F64: "f64", H.F32: "f32", H.F64_IEEE: "f64_ieee"}[vcode],
                                                     name))})
            if v["kernel"] == "k_slab3d":  # the work split the refinement's autotuner picked
                variants[-1]["slab_z_ranges_per_macro"] = v["M"].autotune_choice(v["L"], vcode)
            if name == WORKLOAD and vcode == H.F64_IEEE:
                # the native fp64 apply is bound by the fp64 pipe: 7 fp64
                # operations per macro-interior point (one multiply, three
                # adds of opposite neighbours, three FMAs) against the fp64
                # peak of the GB300 (1.25 TFLOP/s dense = 625 G FMA/s)
                ops = 7.0 * v["interior"]
                achieved = ops / (rv["interior_ms"] * 1e-3) / 1e9
                line["roofline_native_fp64"] = {
                    "bound": "alu", "kernel": f"{v['kernel']} (f64_ieee)", "achieved": achieved,
                    "peak": FP64_PEAK_GOPS, "unit": "G fp64 ops/s", "frac": achieved / FP64_PEAK_GOPS,
                    "peak_kind": "nominal dense fp64 (1.25 TFLOP/s / 2 flops per FMA)",
                    "ops_per_launch": ops, "interior_ms": rv["interior_ms"],
                    "traffic": variants[-1]["traffic"],
                    "GDoF_per_s": variants[-1]["value"],
                    "hbm_frac": variants[-1]["interior_frac"]}
            del v
            torch.cuda.empty_cache()
        line["variants"] = variants
        # latency of one small apply (2 macros, level 7, 16,641 DoFs, L2-resident):
        # the mean event time over back-to-back applies
        v = setup("square2_L7", device, H.F64)
        rv = timed_applies(v, 200, args.warmup, stream)
        line["latency_small"] = {"workload": describe("square2_L7", v["ng"], v["ns"]),
                                 "us_per_apply": 1e3 * rv["total_ms"] / 200,
                                 "us_per_apply_graph_replay": graph_replay_us(v, 200, stream),
                                 "dtype": "f64 data, float-float arithmetic",
                                 "note": "us_per_apply: back-to-back hyteg_apply_timed calls from Python (the host "
                                         "loop bounds it); graph replay: one apply captured in a CUDA graph and "
                                         "replayed, the device-side time per apply"}
        line["batched_small"] = batched_small(v, 64, stream)
        del v

    if rank == 0 and world == 1 and not args.no_variants:
        line["solve"] = solve_workload(device, stream)
        line["group_solve"] = group_workload(device, stream)
        torch.cuda.empty_cache()

    if rank == 0 and world == 1 and not args.no_variants and args.serve_requests > 0:
        line["serving"] = serve_workload(args.serve_requests, args.serve_workers)
        # the same stream with float64 V-cycles: the plain float64 multigrid
        # the mixed-precision server is compared with
        line["serving_fp64_cycles"] = serve_workload(args.serve_requests, args.serve_workers,
                                                     mode=H.SOLVE_F64)
        # below capacity: the same stream offered at 25 % and 50 % of the
        # measured solves/s, so that latency shows service rather than queueing
        cap = line["serving"]["solves_per_s"]
        n_low = min(args.serve_requests, 256)
        line["serving_load_levels"] = [
            {k: v for k, v in serve_workload(n_low, args.serve_workers, rate=f * cap).items() if k != "workload"}
            | {"load_fraction": f} for f in (0.25, 0.5)]

    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == WORKLOAD:
        r = cpu_oracle_run(10, 2)
        ng = r["n_global"]
        line["cpu_baseline"] = {"value": ng / min(r["all_core_s"]) / 1e9, "unit": UNIT, "cores": r["cores"],
                                "kind": "oracle", "sample": r["sample"] + "; best of 10",
                                "single_thread": ng / min(r["one_core_s"]) / 1e9,
                                "scipy_single_thread": ng / min(r["scipy_one_core_s"]) / 1e9}

    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
