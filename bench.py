#!/usr/bin/env python
"""Benchmark of the CPR-preconditioned FGMRES solve phase on B300.

One step = one Newton linear system of a drifting Jacobian sequence on the
128x128x32 synthetic black-oil workload (524,297 3x3 block rows, 9 wells):
cpr_update(A^(k)) (Alg. 3 decides setup or reuse, mu = 30) followed by
cpr_solve(b^(k)) to rtol 1e-6 (FGMRES(30) with CPR).  The Jacobians and
right-hand sides of the sequence are resident in HBM before timing starts.
`value` is FP32-preconditioner solves/s (FP64 outer FGMRES); the FP64 arm is
reported beside it.  Prints one JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
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

import blackoil_synth as bs  # noqa: E402

METRIC = "CPR solves/s & V-cycle HBM GB/s at rtol 1e-6, FP32-precond vs FP64; p50/p99 ms"
UNIT = "solves/s"
WORKLOAD = "128x128x32"
NSEQ = 4            # Jacobians of the drifting sequence kept resident in HBM
RTOL = 1e-6
MU = 30

# DRAM bytes of one launch (dram__bytes_read.sum + dram__bytes_write.sum) of a
# kernel the line rates, from one ncu capture of the build named, at the
# workload named; a kernel changed since then has no entry (traffic null).
NCU_TRAFFIC = {
    ("k_smooth_color", "128x128x32"): {"bytes": 2.5246e6,
                                       "source": "mean DRAM bytes of the 56 color launches of one eager V-cycle, "
                                                 "ncu capture of the commit 1246587 build, cold caches"},
    ("k_sell_spmv", "128x128x32"): {"bytes": 302.96e6 + 10.15e6,
                                    "source": "ncu capture of one k_sell_spmv launch of the commit 1298109 build"},
}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [l.strip().split(", ") for l in open(self.f.name) if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ byte models

def vcycle_bytes(levels, sv, pre=1, post=1):
    """Algorithmic bytes of one V(pre,post) cycle: each level's matrix read once
    per sweep and once for the residual, R and P read once, ~13 vector passes
    per level, the coarsest dense inverse once."""
    tot = 0
    for lv in levels[:-1]:
        tot += (pre + post + 1) * lv["nnz"] * (sv + 4) + 2 * lv["nnz_p"] * (sv + 4)
        tot += 13 * lv["n"] * sv + (pre + post) * lv["n"] * 4
    nL = levels[-1]["n"]
    tot += 8 * nL * nL + 2 * nL * sv
    return tot


def bilu_bytes(nb, nnzb, sv):
    """L and U blocks (9 values + a column index each), D^-1, row pointers and
    color lists, and the vector passes of the forward and backward sweeps."""
    return (nnzb - nb) * (9 * sv + 4) + nb * 9 * sv + 16 * nb + 6 * 3 * nb * sv + nb * sv + 24 * nb


def smooth0_bytes(level, sv, pre=1, post=1):
    """Mean algorithmic bytes of one k_smooth_color launch on the finest level:
    per row of the color its row pointer, b, 1/a_ii and the staged result; per
    off-diagonal entry its column, value and the gathered x; plus the commit of
    the previous color's staged rows (read staged, write x).  Averaged over the
    launches of a V(pre,post) cycle: pre-sweeps ascend the colors (the very first
    color is a separate from-zero kernel), post-sweeps descend, and the first
    post-sweep color has nothing staged to commit."""
    rp, color = level["rowptr"], level["color"]
    off = np.diff(rp) - 1
    nc = int(color.max()) + 1
    rows = np.bincount(color, minlength=nc)
    nnz = np.bincount(color, weights=off, minlength=nc)
    sweeps = [(list(range(nc)), k == 0) for k in range(pre)] + \
             [(list(range(nc - 1, -1, -1)), False) for _ in range(post)]
    launches, prev = [], None
    for si, (cols, from_zero) in enumerate(sweeps):
        if si == pre:
            prev = None                      # the residual kernel committed the pre-sweep's last color
        for t, c in enumerate(cols):
            if from_zero and t == 0:
                prev = c
                continue
            by = rows[c] * (4 + 3 * sv) + nnz[c] * (4 + 2 * sv)
            if prev is not None:
                by += rows[prev] * 2 * sv
            launches.append(by)
            prev = c
    return float(np.mean(launches))


def smooth_color_bytes(levels, sv, pre=1, post=1):
    """Algorithmic bytes and launch count of the k_smooth_color launches of one
    V(pre,post) cycle, all smoothed levels: smooth0_bytes' model per launch
    (row pointer, b, 1/a_ii and staged result per row; column, value and
    gathered x per off-diagonal entry; the previous color's commit)."""
    tot, n = 0.0, 0
    for lv in levels[:-1]:
        if lv.get("color") is None:
            continue
        per = smooth0_bytes(lv, sv, pre, post)
        nlaunch = pre * lv["ncolors"] - 1 + post * lv["ncolors"]   # the very first color is fused elsewhere
        tot += per * nlaunch
        n += nlaunch
    return tot, n


def spmv_bytes(nb, nnzb):
    """FP64 BSR: 72 B of values + 4 B of column per block; x, y and rowptr per block row."""
    return 76 * nnzb + 52 * nb


def cgs_bytes(N, cycles_steps):
    """Dots over j+1 basis vectors and w, then w -= V h: (2j+5) N doubles at step j."""
    return sum(8 * N * (2 * j + 5) for k in cycles_steps for j in range(k))


def cycle_steps(iters, m):
    out = []
    while iters > 0:
        out.append(min(iters, m))
        iters -= m
    return out


# ------------------------------------------------------------------ helpers

def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=world)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def host_sequence(seed_offset=0):
    g = bs.CONFIGS[WORKLOAD]
    if seed_offset:
        import dataclasses
        g = dataclasses.replace(g, seed=g.seed + seed_offset)
    return list(bs.jacobian_sequence(g, NSEQ, drift=0.05))


# --------------------------------------------------------------- our arm

def theta_sweep(cpr, torch, J, stream, thetas=(0.0, 0.05, 0.1, 0.2, 0.3, 0.5)):
    """The Eq. 5.1 threshold of the smoother's coloring (FP32 mode): per theta
    and per coloring (JP, and the paper's Alg. 4-5 on every level of at most
    16384 rows), the colors of every smoothed level, the in-graph V-cycle and
    per-level pre+post smoothing times, one solve's iterations and time, and
    the setup time.  theta and the coloring change only the smoother; the AMG
    hierarchy is the same."""
    class DJ:
        nb = J.nb
        rowptr = torch.from_numpy(J.rowptr).cuda()
        col = torch.from_numpy(J.col).cuda()
        val = torch.from_numpy(J.val).cuda()

    b = torch.from_numpy(J.b).cuda()
    out = []
    for th in thetas:
        for coloring in (0, 1):
            g = cpr.Solver(DJ, precond_fp32=1, theta_color=th, coloring=coloring, coloring_rows=16384,
                           stream=stream.cuda_stream)
            _, st = g.solve(b, rtol=RTOL)          # first solve: captures the step graphs
            x = torch.zeros_like(b)
            _, st = g.solve(b, x, rtol=RTOL)
            parts = g.profile_vcycle_levels(20)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.update(DJ)                           # same pattern, It > mu: a full setup
            torch.cuda.synchronize()
            setup_ms = 1000 * (time.perf_counter() - t0)
            out.append({"theta": th, "coloring": "alg45" if coloring else "jp",
                        "colors": [g.level(l)["ncolors"] for l in range(g.nlev - 1)],
                        "rows": [g.level(l)["n"] for l in range(g.nlev - 1)],
                        "vcycle_us": parts["vcycle_us"],
                        "smooth_us": [p["pre"] + p["post"] for p in parts["levels"]],
                        "iters": st["iters"], "solve_ms": st["solve_ms"], "setup_ms": setup_ms,
                        "converged": st["converged"]})
            g.close()
    return {"workload": f"{WORKLOAD}, FP32 preconditioner, rtol {RTOL}", "rows": out}


def setup_profile(cpr, torch, seq, stream, warm=8):
    """Setup alone (FP32 mode) as the timed step runs it: one handle with
    mu = 0, so that every cpr_update of the drifting sequence is a full setup;
    `warm` updates timed on the host (synchronised), then one more bracketed
    by cudaProfilerStart/Stop (ncu --profile-from-start off) and recorded by
    the setup's phase clock (CPR_SETUP_TIMING: per mark, host and device ms;
    the marks add their own event records, so that setup runs longer)."""
    class DJ:
        def __init__(self, J):
            self.nb = J.nb
            self.rowptr = torch.from_numpy(J.rowptr).cuda()
            self.col = torch.from_numpy(J.col).cuda()
            self.val = torch.from_numpy(J.val).cuda()

    dev = [DJ(J) for J in seq]
    solver = cpr.Solver(dev[0], precond_fp32=1, mu=0, stream=stream.cuda_stream)
    walls = []
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    for k in range(warm):
        torch.cuda.synchronize()
        t = time.perf_counter()
        solver.update(dev[(k + 1) % len(dev)])
        torch.cuda.synchronize()
        walls.append((time.perf_counter() - t) * 1e3)
    os.environ["CPR_SETUP_TIMING"] = "1"
    launches0 = cpr.launch_count()
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    t = time.perf_counter()
    solver.update(dev[(warm + 1) % len(dev)])
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t) * 1e3
    torch.cuda.profiler.stop()
    del os.environ["CPR_SETUP_TIMING"]
    launches = cpr.launch_count() - launches0
    clocks = clk.stop()
    solver.close()
    return {"workload": f"{WORKLOAD} FP32-mode setup through cpr_update (mu = 0)", "clocks": clocks,
            "warm_wall_ms": walls,
            "warm_wall_ms_median": statistics.median(walls[len(walls) // 2:]),
            "profiled_wall_ms": wall, "launches": launches}


def resetup_profile(cpr, torch, seq, stream, updates=4):
    """The numeric-only resetup (resetup = 1, FP32 mode) alone: a setup on the
    sequence's first Jacobian, then `updates` rebuilds on the next ones (the
    first captures the refresh graph, the rest replay it), each inside the
    library's NVTX range "numeric refresh" (ncu --nvtx-include)."""
    class DJ:
        def __init__(self, J):
            self.nb = J.nb
            self.rowptr = torch.from_numpy(J.rowptr).cuda()
            self.col = torch.from_numpy(J.col).cuda()
            self.val = torch.from_numpy(J.val).cuda()

    dev = [DJ(J) for J in seq]
    solver = cpr.Solver(dev[0], precond_fp32=1, mu=0, resetup=1, stream=stream.cuda_stream)
    walls = []
    for k in range(1, updates + 1):
        torch.cuda.synchronize()
        t = time.perf_counter()
        solver.update(dev[k % len(dev)])
        torch.cuda.synchronize()
        walls.append((time.perf_counter() - t) * 1e3)
    solver.close()
    return {"workload": f"{WORKLOAD} FP32-mode numeric resetup", "update_wall_ms": walls}


def vcycle_profile(cpr, torch, workload, stream):
    """One FP32 hierarchy of `workload`: the in-graph time of every V-cycle
    part (20 repetitions per graph) and the level-0 smoothing colors' rows,
    entries and algorithmic bytes; then one eager V-cycle (cpr_vcycle)
    bracketed by cudaProfilerStart/Stop for a one-kernel ncu capture."""
    J = bs.jacobian(bs.CONFIGS[workload])

    class DJ:
        nb = J.nb
        rowptr = torch.from_numpy(J.rowptr).cuda()
        col = torch.from_numpy(J.col).cuda()
        val = torch.from_numpy(J.val).cuda()

    b = torch.from_numpy(J.b).cuda()
    g = cpr.Solver(DJ, precond_fp32=1, stream=stream.cuda_stream)
    _, st = g.solve(b, rtol=RTOL)
    parts = g.profile_vcycle_levels(20)
    lv0 = g.level(0)
    color, rp = lv0["color"], lv0["rowptr"]
    off = np.diff(rp) - 1
    nc = int(color.max()) + 1
    rows = np.bincount(color, minlength=nc)
    ents = np.bincount(color, weights=off, minlength=nc)
    per_color = [{"rows": int(rows[c]), "offdiag": int(ents[c]),
                  "bytes": int(rows[c] * (4 + 3 * 4) + ents[c] * (4 + 2 * 4))} for c in range(nc)]
    bp = torch.from_numpy(np.random.default_rng(1).standard_normal(J.nb)).cuda()
    xp = torch.zeros_like(bp)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    g.vcycle(bp, xp)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    levels = [{k: g.level(l)[k] for k in ("n", "nnz", "ncolors")} for l in range(g.nlev)]
    g.close()
    return {"workload": f"{workload}, FP32 preconditioner", "iters": st["iters"], "levels": levels,
            "vcycle_parts_us": parts, "level0_colors": per_color,
            "note": "bytes: per row its row pointer, b, 1/a_ii and the staged result; per off-diagonal "
                    "entry its column, value and the gathered x (FP32)"}


def run_arm(cpr, torch, seq_dev, rhs_dev, fp32, K, W, world, stream, profile_region=False):
    """Time K update+solve steps of one precision arm; returns a dict."""
    S = len(seq_dev)
    solver = cpr.Solver(seq_dev[0], precond_fp32=int(fp32), mu=MU, stream=stream.cuda_stream)
    x = torch.zeros_like(rhs_dev[0])
    stats = []

    def step(k):
        if k:
            solver.update(seq_dev[k % S])
        with torch.cuda.stream(stream):
            x.zero_()
        _, st = solver.solve(rhs_dev[k % S], x, rtol=RTOL)
        if not st["converged"]:
            raise RuntimeError(f"solve did not converge: {st}")
        return st

    for k in range(W):
        step(k)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    launches0 = cpr.launch_count()
    barrier(world)
    torch.cuda.synchronize()
    if profile_region:
        torch.cuda.profiler.start()
    ev[0].record(stream)
    for i in range(K):
        stats.append(step(W + i))
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    if profile_region:
        torch.cuda.profiler.stop()
    barrier(world)
    launches = cpr.launch_count() - launches0
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(K)]
    total = ev[0].elapsed_time(ev[K])
    # Per-family times: a second timed region of the same steps with CUDA-event
    # brackets around each family (the brackets add event nodes to the step
    # graphs, so the headline above is taken without them).
    P = min(K, 4)
    outer = [cpr.PROF_SPMV, cpr.PROF_VCYCLE, cpr.PROF_BILU, cpr.PROF_CGS, cpr.PROF_RESID2]
    solver.profile(True, outer)
    pe = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    pe[0].record(stream)
    for i in range(P):
        step(W + K + i)
    pe[1].record(stream)
    torch.cuda.synchronize()
    fam = {f: solver.profile_read(f) for f in outer}
    prof_ms = pe[0].elapsed_time(pe[1]) / P
    # the level-0 color sweeps sit inside the V-cycle bracket: a pass of their own
    solver.profile(True, [cpr.PROF_SMOOTH0])
    for i in range(P):
        step(W + K + P + i)
    torch.cuda.synchronize()
    fam[cpr.PROF_SMOOTH0] = solver.profile_read(cpr.PROF_SMOOTH0)
    solver.profile(False)
    levels = [solver.level(l) for l in range(solver.nlev)]
    # in-graph device time of each V-cycle part (between solves)
    parts = solver.profile_vcycle_levels(20)
    for l, d in enumerate(parts["levels"]):
        d.update(n=levels[l]["n"], nnz=levels[l]["nnz"], ncolors=levels[l]["ncolors"])
    solver.close()
    return {"per_ms": per, "total_ms": total, "stats": stats, "fam": fam, "levels": levels,
            "launches": launches, "profiled_ms_per_step": prof_ms, "profiled_steps": P, "parts": parts}


def option_arm(cpr, torch, seq_dev, rhs_dev, K, W, stream, note, **opts):
    """The headline's update+solve steps with extra solver options, in both
    precisions."""
    S = len(seq_dev)
    out = {}
    for name, fp32 in (("fp32", 1), ("fp64", 0)):
        solver = cpr.Solver(seq_dev[0], precond_fp32=fp32, mu=MU, stream=stream.cuda_stream, **opts)
        x = torch.zeros_like(rhs_dev[0])
        stats = []

        def step(k):
            if k:
                solver.update(seq_dev[k % S])
            with torch.cuda.stream(stream):
                x.zero_()
            _, st = solver.solve(rhs_dev[k % S], x, rtol=RTOL)
            if not st["converged"]:
                raise RuntimeError(f"solve did not converge: {st}")
            return st

        for k in range(W):
            step(k)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        for i in range(K):
            stats.append(step(W + i))
        ev[1].record(stream)
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1])
        nlev = solver.bilu()[1]
        solver.close()
        out[name] = {"value": K / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / K,
                     "iters_mean": statistics.mean(st["iters"] for st in stats),
                     "setup_ms_mean": statistics.mean([st["setup_ms"] for st in stats if st["setup_called"]]
                                                      or [0.0]),
                     "solve_phase_ms_mean": statistics.mean(st["solve_ms"] for st in stats),
                     "setups": sum(st["setup_called"] for st in stats), "bilu_colors": nlev}
    out["note"] = f"{K} timed steps after {W} warm-up, same sequence and rule as the headline; {note}"
    return out


def e2e_arm(cpr, torch, seq_host, K, W, stream):
    """Same metric through the C ABI with pinned HOST buffers (copies inside the calls)."""
    S = len(seq_host)

    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.from_numpy(a[:1]).dtype, pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()

    hseq = []
    for J in seq_host:
        hseq.append(bs.Jacobian(J.nb, pinned(J.rowptr), pinned(J.col), pinned(J.val), pinned(J.b)))
    xh = pinned(np.zeros(3 * seq_host[0].nb))
    solver = cpr.Solver(hseq[0], precond_fp32=1, mu=MU, stream=stream.cuda_stream)

    def step(k):
        # a Newton sequence keeps A's block pattern: each step hands the library
        # the new values (cpr_update_values), as a simulator's Newton loop would
        if k:
            solver.update_values(hseq[k % S].val)
        xh[...] = 0.0
        _, st = solver.solve(hseq[k % S].b, xh, rtol=RTOL)
        return st

    for k in range(W):
        step(k)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(K):
        step(W + i)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    solver.close()
    J = seq_host[0]
    h2d = J.val.nbytes + J.b.nbytes + xh.nbytes
    return {"value": K / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "calls": "cpr_update_values(values), then cpr_solve(b, x) with pinned host buffers",
            "d2h_bytes_per_step": int(xh.nbytes)}


def batched_arm(cpr, torch, K, stream, nsys=64):
    """64 independent systems (16^3 .. 64x64x16): one batched FP32-preconditioner
    solve, timed with the fixed lanes-per-row rule and again after the
    schedule autotuner (cpr_autotune) ran on the batch's hierarchy, vs the same
    systems solved one after another with plain FP64 CPR."""
    specs = bs.batch_specs(nsys)
    Js = [bs.jacobian(g) for g in specs]

    class DJ:
        def __init__(self, J):
            self.nb = J.nb
            self.rowptr = torch.from_numpy(J.rowptr).cuda()
            self.col = torch.from_numpy(J.col).cuda()
            self.val = torch.from_numpy(J.val).cuda()

    dj = [DJ(J) for J in Js]
    bvec = [torch.from_numpy(J.b).cuda() for J in Js]
    bt = cpr.BatchSolver(dj, precond_fp32=1, mu=MU, stream=stream.cuda_stream)
    xs = [torch.zeros_like(b) for b in bvec]
    for _ in range(2):
        bt.solve(bvec, xs, rtol=RTOL)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed():
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(K):
            for x in xs:
                x.zero_()
            _, sts_ = bt.solve(bvec, xs, rtol=RTOL)
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / K, sts_

    ms_rule, _ = timed()          # the fixed lanes-per-row rule
    rule = [bt.schedule(l) for l in range(bt.nlev - 1)]
    t0 = time.perf_counter()
    bp_before, bp_after = bt.autotune(reps=10)
    tune_ms = 1000 * (time.perf_counter() - t0)
    bt.solve(bvec, xs, rtol=RTOL)  # recaptures the step graphs with the tuned schedule
    ms, sts = timed()
    tuned = [bt.schedule(l) for l in range(bt.nlev - 1)]
    ok = all(st["converged"] for st in sts)
    iters = [st["iters"] for st in sts]
    # Alg. 3 on a batch compares the largest step count with mu: the system
    # that took it decides whether the next batch update rebuilds B
    forcing = int(np.argmax(iters))
    bt.close()
    # the same systems, one handle each, FP64 preconditioner, solved in turn
    singles = [cpr.Solver(d, precond_fp32=0, mu=MU, stream=stream.cuda_stream) for d in dj]
    for sv, b, x in zip(singles, bvec, xs):
        x.zero_()
        sv.solve(b, x, rtol=RTOL)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(max(1, K // 2)):
        for sv, b, x in zip(singles, bvec, xs):
            x.zero_()
            sv.solve(b, x, rtol=RTOL)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_seq = ev0.elapsed_time(ev1) / max(1, K // 2)
    for sv in singles:
        sv.close()
    cells = sum(g.ncells for g in specs)
    return {"workload": f"{nsys} systems, 16^3..64x64x16 cells ({cells} cells), FP32 preconditioner",
            "value": nsys / (ms / 1000.0), "unit": UNIT, "ms_per_batch": ms, "all_converged": ok,
            "autotune": {"schedule": tuned, "fixed_rule_schedule": rule, "tuning_ms": tune_ms,
                         "fixed_rule_value": nsys / (ms_rule / 1000.0), "fixed_rule_ms_per_batch": ms_rule,
                         "gain_over_fixed_rule": ms_rule / ms,
                         "pressure_cycle_us_before": bp_before, "pressure_cycle_us_after": bp_after},
            "iters_max": max(iters), "iters_mean": statistics.mean(iters),
            "alg3": {"deciding_system": forcing, "deciding_iters": iters[forcing], "mu": MU,
                     "next_update_rebuilds": iters[forcing] > MU},
            "fp64_one_by_one": {"value": nsys / (ms_seq / 1000.0), "unit": UNIT, "ms": ms_seq},
            "speedup_vs_fp64_one_by_one": ms_seq / ms}


def serve_arm(full: bool):
    """Continuous-batching service: 32 ensemble members x 5 drifting Newton
    Jacobians, Poisson arrivals at 200 requests/s, 16 slots, resident
    hierarchies with the adaptive rule per member, FP32 preconditioner; beside
    it the same requests served one at a time by plain FP64 CPR (setup every
    request, mu = 0)."""
    from paper_2201_01970_b300 import serve
    members = bs.ensemble_specs(32, full=full)
    reqs = serve.poisson_requests(members, steps=5, rate=200.0, seed=0)
    for r in reqs:          # the payloads arrive in page-locked receive buffers
        serve.pin_request(r)
    # 16 concurrent solves driven by one polling thread, first setups on 4
    # helper threads: the best of a sweep over 16/24/32 slots and 4/8/16
    # helpers on this ensemble (throughput ~169/s in every case that kept up;
    # p99 lowest with 16 and 4)
    srv = serve.Server(slots=16, setup_workers=4, precond_fp32=1, mu=MU)
    m = srv.run(reqs, realtime=True)
    srv.close()
    ok = all(r.stats.get("converged") for r in reqs)
    # capacity: the same requests all queued at once, so the loop never waits
    # for an arrival (same slots, helpers and member order)
    sat = [serve.Request(r.member, r.step, r.A, r.b, 0.0, same_pattern=r.same_pattern) for r in reqs]
    srv = serve.Server(slots=16, setup_workers=4, precond_fp32=1, mu=MU)
    ms = srv.run(sat, realtime=False)
    srv.close()
    ok = ok and all(r.stats.get("converged") for r in sat)
    base = [serve.Request(r.member, r.step, r.A, r.b, r.arrival, same_pattern=r.same_pattern) for r in reqs]
    srv = serve.Server(slots=1, precond_fp32=0, mu=0)
    mb = srv.run(base, realtime=False)
    srv.close()
    cells = sum(g.ncells for g in members)
    m.update({"workload": f"32 members ({'32x32x8..128x128x32' if full else '32x32x8..64x64x16'}, "
                          f"{cells} cells), 5 Newton steps each, Poisson 200/s",
              "all_converged": ok,
              "capacity": {"value": ms["value"], "unit": "solves/s", "makespan_s": ms["makespan_s"],
                           "note": "the same requests all queued at time 0: throughput when the loop never "
                                   "waits for an arrival"},
              "plain_fp64_cpr_serial": {"value": mb["value"], "unit": "solves/s", "p50_ms": mb["p50_ms"],
                                        "p99_ms": mb["p99_ms"]}})
    return m


def adaptive_sweep(cpr, torch, stream, mus=(0, 10, 20, 30, 40, 50, 60, 100), nseq=10):
    """Alg. 3 on a 10-Jacobian drifting Newton sequence of the 60x220x85 banded
    workload, per threshold mu and per preconditioner precision: total device
    time of the sequence (update + solve per step; the first setup, done at
    construction, is outside the timed region for every mu alike), setups
    taken and iterations per step."""
    g = bs.CONFIGS["60x220x85"]
    seq = list(bs.jacobian_sequence(g, nseq, drift=0.05))

    class DJ:
        def __init__(self, J):
            self.nb = J.nb
            self.rowptr = torch.from_numpy(J.rowptr).cuda()
            self.col = torch.from_numpy(J.col).cuda()
            self.val = torch.from_numpy(J.val).cuda()

    dev = [DJ(J) for J in seq]
    rhs = [torch.from_numpy(J.b).cuda() for J in seq]
    x = torch.zeros_like(rhs[0])
    runs = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def one(fp32, mu):
        s = cpr.Solver(dev[0], precond_fp32=int(fp32), mu=mu, stream=stream.cuda_stream)
        sts = []
        torch.cuda.synchronize()
        ev0.record(stream)
        for k in range(nseq):
            if k:
                s.update(dev[k])
            with torch.cuda.stream(stream):
                x.zero_()
            _, st = s.solve(rhs[k], x, rtol=RTOL)
            sts.append(st)
        ev1.record(stream)
        torch.cuda.synchronize()
        s.close()
        return ev0.elapsed_time(ev1), sts

    one(True, 0)                                  # warm-up: pool, graphs, first-touch
    for fp32 in (True, False):
        for mu in mus:
            ms, sts = one(fp32, mu)
            runs.append({"precond": "fp32" if fp32 else "fp64", "mu": mu, "total_ms": ms,
                         "ms_per_step": ms / nseq,
                         "setups": int(sum(st["setup_called"] for st in sts[1:])),
                         "iters": [st["iters"] for st in sts],
                         "all_converged": all(st["converged"] for st in sts)})
    return {"workload": f"60x220x85 banded, {nseq}-Jacobian drifting sequence, rtol {RTOL}",
            "nb": seq[0].nb, "nnzb": seq[0].nnzb, "runs": runs}


def host_cpu():
    """(logical CPUs, CPU model) of this host."""
    model = "unknown"
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return os.cpu_count() or 1, model


def cpu_baseline(seq_host, omp_samples=5):
    """The FP64 oracle on the host, in the two forms of the CPU baseline: the
    single-threaded build (one update+solve: the full setup, as It > mu, then
    the solve) and the OpenMP build over every host core (rows within a color,
    SpMV rows, vector updates; bit-identical results), median of
    `omp_samples` update+solves of the sequence.  Setup and solve are timed
    separately.  Returns the line's object and the OpenMP solution of the
    sequence's second Jacobian (for the error of the GPU solutions)."""
    import oracle
    nproc, model = host_cpu()
    S = len(seq_host)
    o = oracle.Solver(seq_host[0], mu=MU)
    t0 = time.perf_counter()
    o.update(seq_host[1])
    t1 = time.perf_counter()
    _, st1 = o.solve(seq_host[1].b, rtol=RTOL)
    t2 = time.perf_counter()
    o.close()
    single = {"value": 1.0 / (t2 - t0), "unit": UNIT, "cores": 1, "setup_s": t1 - t0, "solve_s": t2 - t1,
              "iters": st1["iters"], "samples": 1}
    p = oracle.Solver(seq_host[0], mu=MU, omp=True)
    threads = oracle.threads(True)
    setups, solves, x_ref, iters = [], [], None, []
    for k in range(omp_samples):
        J = seq_host[1 + k % (S - 1)]
        t0 = time.perf_counter()
        p.update(J)
        t1 = time.perf_counter()
        x, st = p.solve(J.b, rtol=RTOL)
        t2 = time.perf_counter()
        if not st["setup_called"]:
            raise RuntimeError("the CPU baseline's update kept B; every timed step must set up")
        setups.append(t1 - t0)
        solves.append(t2 - t1)
        iters.append(st["iters"])
        if k == 0:
            x_ref = x
    p.close()
    tot = [a + b for a, b in zip(setups, solves)]
    med = statistics.median(tot)
    out = {"value": 1.0 / med, "unit": UNIT, "cores": threads, "kind": "oracle",
           "nproc": nproc, "cpu_model": model,
           "sample": f"OpenMP oracle, median of {omp_samples} update+solves (full setup each, It > mu) "
                     f"of the {WORKLOAD} sequence; single-threaded oracle: one update+solve",
           "setup_s_median": statistics.median(setups), "solve_s_median": statistics.median(solves),
           "iters": iters, "single_thread": single,
           "paper_context": "paper (Xeon 8260 / Tesla T4, SPE10 3P): over 6.5x with 16 OpenMP threads, "
                            "over 9.5x in CUDA, each against one thread"}
    return out, x_ref


def gpu_error_vs_oracle(cpr, torch, J_dev, J, x_ref, stream):
    """Relative error, against the FP64 oracle's solution x_ref, of the GPU
    solutions of the same Jacobian from zero to rtol (fresh handles, so B is
    built from this Jacobian on both sides), in both preconditioner precisions."""
    out = {}
    b = torch.from_numpy(J.b).cuda()
    for name, fp32 in (("fp32", 1), ("fp64", 0)):
        s = cpr.Solver(J_dev, precond_fp32=fp32, mu=MU, stream=stream.cuda_stream)
        x = torch.zeros_like(b)
        _, st = s.solve(b, x, rtol=RTOL)
        torch.cuda.synchronize()
        xg = x.cpu().numpy()
        s.close()
        out[name] = {"rel_error": float(np.linalg.norm(xg - x_ref) / np.linalg.norm(x_ref)),
                     "iters": st["iters"]}
    out["note"] = ("||x_gpu - x_oracle|| / ||x_oracle|| on the sequence's second Jacobian, both solved "
                   f"from zero to rtol {RTOL} with B built from that Jacobian")
    return out


# ---------------------------------------------------------- reference arm

def reference_arm(args, rank, world):
    """The FP64 oracle as the reference implementation, on the host cores (its
    OpenMP build, bit-identical to the single-threaded one).  Each step is one
    update+solve of the workload's drifting sequence, as in our arm.  The first
    warm-up step is timed: when all K+W steps of the full workload would not
    end within the budget, every step runs on a z-slab of the workload (the
    first nz' layers, same generator) instead, reported as that slab with its
    own measured times (nothing is scaled)."""
    if rank != 0:
        return
    import dataclasses
    import oracle
    budget = 200.0
    g = bs.CONFIGS[WORKLOAD]
    nsteps = args.steps + args.warmup

    def run(gs, first_only=False):
        seq = list(bs.jacobian_sequence(gs, NSEQ, drift=0.05))
        o = oracle.Solver(seq[0], mu=MU, omp=True)
        times = []
        for k in range(1 if first_only else nsteps):
            J = seq[(k + 1) % NSEQ]
            t0 = time.perf_counter()
            o.update(J)
            _, st = o.solve(J.b, rtol=RTOL)
            times.append(time.perf_counter() - t0)
        o.close()
        return times

    t_first = run(g, first_only=True)[0]
    gs = g
    if t_first * nsteps > budget:
        nz = max(1, int(g.nz * budget / (t_first * nsteps)))
        gs = dataclasses.replace(g, nz=nz)
    times = run(gs)[args.warmup:]
    per = statistics.mean(times)
    value = 1.0 / per
    nproc, model = host_cpu()
    threads = oracle.threads(True)
    wl = (f"{WORKLOAD} synthetic black-oil, drifting Newton sequence" if gs is g else
          f"{g.nx}x{g.ny}x{gs.nz} z-slab of the {WORKLOAD} workload (the full grid would not fit "
          f"{nsteps} steps in {budget:.0f} s: {t_first:.1f} s per step)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * per,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl, "mu": MU, "rtol": RTOL, "restart": 30},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "nproc": nproc, "cpu_model": model,
                             "sample": f"each step one update+solve of the {wl} (OpenMP oracle, "
                                       f"{threads} threads); first full-size step {t_first:.2f} s"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-bilu-natural", action="store_true",
                    help="skip the level-scheduled (natural-order) BILU(0) line")
    ap.add_argument("--theta-sweep", action="store_true",
                    help="only sweep the smoother coloring's Eq. 5.1 threshold: colors, V-cycle time, iterations")
    ap.add_argument("--setup-profile", action="store_true",
                    help="only time setups of the workload, the last one bracketed for ncu and phase-marked")
    ap.add_argument("--resetup-profile", action="store_true",
                    help="only run numeric-only resetups of the workload (NVTX range 'numeric refresh')")
    ap.add_argument("--no-resetup-numeric", action="store_true",
                    help="skip the numeric-only resetup line")
    ap.add_argument("--no-ua-amg", action="store_true",
                    help="skip the UA-AMG (amg = 1) line")
    ap.add_argument("--no-adaptive", action="store_true",
                    help="skip Alg. 3 on the 60x220x85 drifting sequence (mu = 0, 30, 60) in the line")
    ap.add_argument("--no-alg45", action="store_true",
                    help="skip the Alg. 4-5 coloring (coloring = 1) line")
    ap.add_argument("--serve-scaled", action="store_true",
                    help="serving ensemble over the scaled 32x32x8..64x64x16 range instead of the full "
                         "32x32x8..128x128x32 one")
    ap.add_argument("--arm", default="both", choices=["both", "fp32", "fp64"],
                    help="precision arms to time (the JSON line needs both)")
    ap.add_argument("--vcycle-profile", default=None, metavar="WORKLOAD",
                    help="only time the V-cycle parts of WORKLOAD's FP32 hierarchy and bracket one eager "
                         "V-cycle for ncu")
    ap.add_argument("--serve-only", action="store_true",
                    help="only run the serving arm and print its object")
    ap.add_argument("--adaptive-sweep", action="store_true",
                    help="only run Alg. 3's mu sweep on the 60x220x85 sequence and print it")
    ap.add_argument("--profile-region", action="store_true",
                    help="bracket the first timed region with cudaProfilerStart/Stop (for ncu)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return

    import torch
    import paper_2201_01970_b300 as cpr
    from paper_2201_01970_b300 import build
    if rank == 0:
        build.build()
    barrier(world)
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    if args.adaptive_sweep:
        res = adaptive_sweep(cpr, torch, stream)
        if rank == 0:
            print(json.dumps({"adaptive_sweep": res}), flush=True)
        return
    if args.theta_sweep:
        res = theta_sweep(cpr, torch, bs.jacobian(bs.CONFIGS[WORKLOAD]), stream)
        if rank == 0:
            print(json.dumps({"theta_sweep": res}), flush=True)
        return
    if args.vcycle_profile:
        res = vcycle_profile(cpr, torch, args.vcycle_profile, stream)
        if rank == 0:
            print(json.dumps({"vcycle_profile": res}), flush=True)
        return
    if args.serve_only:
        res = serve_arm(not args.serve_scaled)
        if rank == 0:
            print(json.dumps({"serving": res}), flush=True)
        return
    if args.resetup_profile:
        res = resetup_profile(cpr, torch, host_sequence(), stream)
        if rank == 0:
            print(json.dumps({"resetup_profile": res}), flush=True)
        return
    if args.setup_profile:
        res = setup_profile(cpr, torch, host_sequence(), stream)
        if rank == 0:
            print(json.dumps({"setup_profile": res}), flush=True)
        return

    seq_host = host_sequence(seed_offset=rank)

    class DJ:
        def __init__(self, J):
            self.nb = J.nb
            self.rowptr = torch.from_numpy(J.rowptr).cuda()
            self.col = torch.from_numpy(J.col).cuda()
            self.val = torch.from_numpy(J.val).cuda()

    seq_dev = [DJ(J) for J in seq_host]
    rhs_dev = [torch.from_numpy(J.b).cuda() for J in seq_host]
    torch.cuda.synchronize()
    K, W = args.steps, args.warmup

    clk = ClockSampler(local)
    clk.start()
    pr = args.profile_region
    r32 = r64 = None
    if args.arm in ("both", "fp32"):
        r32 = run_arm(cpr, torch, seq_dev, rhs_dev, True, K, W, world, stream, pr)
        pr = False
    if args.arm in ("both", "fp64"):
        r64 = run_arm(cpr, torch, seq_dev, rhs_dev, False, K, W, world, stream, pr)
    clocks = clk.stop()
    if r32 is None or r64 is None:
        r = r32 or r64
        if rank == 0:
            print(json.dumps({"partial": args.arm, "ms_per_step": r["total_ms"] / K,
                              "launches_per_step": r["launches"] / K,
                              "setup_ms_mean": statistics.mean([st["setup_ms"] for st in r["stats"]
                                                                if st["setup_called"]] or [0.0]),
                              "solve_phase_ms_mean": statistics.mean([st["solve_ms"] for st in r["stats"]]),
                              "iters": [st["iters"] for st in r["stats"]]}), flush=True)
        return

    e2e = None if args.no_e2e else e2e_arm(cpr, torch, seq_host, max(3, K // 2), 1, stream)
    batched = None if args.no_batch else batched_arm(cpr, torch, max(3, K // 2), stream)
    serving = None if args.no_serve else serve_arm(not args.serve_scaled)
    natural = None if args.no_bilu_natural else option_arm(
        cpr, torch, seq_dev, rhs_dev, max(3, K // 3), W, stream,
        "bilu_order = 1: the paper's level-scheduled second stage, one launch per level set", bilu_order=1)
    alg45 = None if args.no_alg45 else option_arm(
        cpr, torch, seq_dev, rhs_dev, K, W, stream,
        "coloring = 1: the paper's Alg. 4-5 grouping on the levels of at most 4096 rows, JP above", coloring=1)
    ua = None if args.no_ua_amg else option_arm(
        cpr, torch, seq_dev, rhs_dev, K, W, stream,
        "amg = 1: the paper's UA-AMG first stage (double pairwise aggregation, handshake rounds with "
        "attachment, unit P) with the nonlinear AMLI-cycle (2 GCR steps per coarse correction)", amg=1)
    # Alg. 3 on the 60x220x85 sequence: mu = 0 and 30 rebuild B every step at
    # this size (every solve takes over 40 inner steps), mu = 60 keeps B^(1)
    adaptive = None if args.no_adaptive else adaptive_sweep(cpr, torch, stream, mus=(0, 30, 60))
    numeric = None if args.no_resetup_numeric else option_arm(
        cpr, torch, seq_dev, rhs_dev, K, W, stream,
        "resetup = 1: each rebuild keeps the first setup's levels, strength sets, C/F splits and colorings "
        "and recomputes the values", resetup=1)
    cpu = err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, x_ref = cpu_baseline(seq_host)
        err = gpu_error_vs_oracle(cpr, torch, seq_dev[1], seq_host[1], x_ref, stream)

    t32 = max_over_ranks(r32["total_ms"], world)
    t64 = max_over_ranks(r64["total_ms"], world)
    value = sum_over_ranks(K, world) / (t32 / 1000.0)
    v64 = sum_over_ranks(K, world) / (t64 / 1000.0)
    if e2e is not None:
        e2e["value"] = sum_over_ranks(e2e["value"], world)

    J0 = seq_host[0]
    nb, nnzb, N = J0.nb, J0.nnzb, 3 * J0.nb
    hbm, peak_kind = peaks()

    def fam_report(r, sv):
        fam, lv = r["fam"], r["levels"]
        out = {}
        n, ms = fam[cpr.PROF_SPMV]
        if n:
            out["spmv"] = {"launches": n, "avg_us": 1000 * ms / n,
                           "gbs": spmv_bytes(nb, nnzb) / (ms / n * 1e-3) / 1e9}
        n, ms = fam[cpr.PROF_VCYCLE]
        if n:
            vb = vcycle_bytes(lv, sv)
            out["vcycle"] = {"applications": n, "avg_us": 1000 * ms / n, "bytes": vb,
                             "gbs": vb / (ms / n * 1e-3) / 1e9}
        n, ms = fam[cpr.PROF_BILU]
        if n:
            bb = bilu_bytes(nb, nnzb, sv)
            out["bilu"] = {"applications": n, "avg_us": 1000 * ms / n, "bytes": bb,
                           "gbs": bb / (ms / n * 1e-3) / 1e9}
        n, ms = fam[cpr.PROF_CGS]
        if n:
            cb = sum(cgs_bytes(N, cycle_steps(st["iters"], 30)) for st in r["stats"])
            out["cgs"] = {"steps": n, "avg_us": 1000 * ms / n, "gbs": cb / (ms * 1e-3) / 1e9}
        n, ms = fam[cpr.PROF_SMOOTH0]
        if n:
            sb = smooth0_bytes(lv[0], sv)
            out["smooth0"] = {"launches": n, "avg_us": 1000 * ms / n, "bytes_per_launch": sb,
                              "gbs": sb / (ms / n * 1e-3) / 1e9}
        n, ms = fam[cpr.PROF_RESID2]
        if n:
            rb = nnzb * (3 * sv + 4) + nb * (4 + 3 * 8 + 3 * sv) + nnzb * sv
            out["resid2"] = {"launches": n, "avg_us": 1000 * ms / n,
                             "gbs": rb / (ms / n * 1e-3) / 1e9}
        return out

    f32 = fam_report(r32, 4)
    f64 = fam_report(r64, 8)
    sm0 = f32.get("smooth0", {})
    sp = f32.get("spmv", {})
    # The outer SpMV is the largest single kernel of the step (launch-list
    # share).  Its roofline is HBM: the algorithmic bytes of one launch,
    # 76 nnzb + 52 nb (FP64 values and column of every block, x, y and the
    # slice offsets), over its live average duration, against the measured
    # copy bandwidth.  B300's FP64 pipe is its other limit (about 91 % busy
    # under ncu), reported beside it: 18 nnzb flops against 296 DFMA
    # thread-instructions per cycle x 2 x the maximum SM clock.
    fp64_peak = 296 * 2 * 2.032e9 / 1e12
    spmv_tflops = (18.0 * nnzb / (sp["avg_us"] * 1e-6) / 1e12) if sp.get("avg_us") else None
    tr = NCU_TRAFFIC.get(("k_sell_spmv", WORKLOAD))
    roof = {"kernel": "k_sell_spmv (outer FP64 SpMV on the sliced-ELL copy, w = A z)", "bound": "hbm",
            "achieved": sp.get("gbs"), "peak": hbm, "unit": "GB/s",
            "frac": (sp.get("gbs") / hbm) if sp.get("gbs") else None,
            "peak_kind": f"{peak_kind} hbm_gbs (of {peak_kind})",
            "bytes_per_launch": spmv_bytes(nb, nnzb), "avg_us": sp.get("avg_us"),
            "traffic": tr["bytes"] if tr else None,
            "traffic_source": tr["source"] if tr else None,
            "fp64_pipe": {"achieved": spmv_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                          "frac": spmv_tflops / fp64_peak if spmv_tflops else None,
                          "flops_per_launch": 18.0 * nnzb,
                          "peak_kind": "FP64 FMA rate x max SM clock (derived from the ncu peak of "
                                       "sm__sass_thread_inst_executed_op_dfma_pred_on)"}}
    roof_sm = {"kernel": "k_smooth_color on the finest pressure level (multi-color GS color sweep, FP32)",
               "bound": "hbm", "achieved": sm0.get("gbs"), "peak": hbm, "unit": "GB/s",
               "frac": (sm0.get("gbs") / hbm) if sm0.get("gbs") else None,
               "peak_kind": f"{peak_kind} hbm_gbs", "traffic": None,
               "bytes_per_launch": sm0.get("bytes_per_launch")}
    # The dominant kernel by launch-list share is the multi-color GS sweep
    # k_smooth_color (its instances over all levels: ~29 % of a step's kernel
    # time).  Its rate: the algorithmic bytes of every color launch of one
    # V(1,1) cycle (smooth_color_bytes) over the live in-graph time of all
    # pre- and post-smoothing sweeps (vcycle_parts_us), against HBM.
    parts32 = r32["parts"]["levels"]
    sweep_us = sum(d["pre"] + d["post"] for d in parts32)
    sweep_bytes, sweep_launches = smooth_color_bytes(r32["levels"], 4)
    tr_sm = NCU_TRAFFIC.get(("k_smooth_color", WORKLOAD))
    roof_family = {"kernel": "k_smooth_color, all levels (multi-color GS color sweeps, FP32; the largest kernel "
                             "family of the step by launch-list share)",
                   "bound": "hbm", "achieved": sweep_bytes / (sweep_us * 1e-6) / 1e9, "peak": hbm, "unit": "GB/s",
                   "frac": sweep_bytes / (sweep_us * 1e-6) / 1e9 / hbm,
                   "peak_kind": f"{peak_kind} hbm_gbs (of {peak_kind})",
                   "bytes_per_launch": sweep_bytes / sweep_launches, "launches_per_vcycle": sweep_launches,
                   "avg_us": sweep_us / sweep_launches,
                   "traffic": tr_sm["bytes"] if tr_sm else None,
                   "traffic_source": tr_sm["source"] if tr_sm else None}

    def pct(a, q):
        return float(np.percentile(np.array(a), q))

    iters32 = [s["iters"] for s in r32["stats"]]
    iters64 = [s["iters"] for s in r64["stats"]]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": t32 / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 preconditioner / f64 outer", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD} synthetic black-oil (3x3 BSR, 9 wells), {NSEQ}-Jacobian "
                               f"drifting Newton sequence resident in HBM, update+solve per step",
                   "nb": nb, "nnzb": nnzb, "dof": N, "mu": MU, "rtol": RTOL, "restart": 30,
                   "l2": "inputs larger than L2 (A values 261 MB per Jacobian)",
                   "parallelism": f"replicas x{world}"},
        "p50_ms": pct(r32["per_ms"], 50), "p99_ms": pct(r32["per_ms"], 99),
        "iters_mean": statistics.mean(iters32),
        "setups_in_timed_region": sum(s["setup_called"] for s in r32["stats"]),
        "setup_ms_mean": statistics.mean([s["setup_ms"] for s in r32["stats"] if s["setup_called"]] or [0.0]),
        "solve_phase_ms_mean": statistics.mean([s["solve_ms"] for s in r32["stats"]]),
        "fp64": {"value": v64, "unit": UNIT, "ms_per_step": t64 / K, "p50_ms": pct(r64["per_ms"], 50),
                 "p99_ms": pct(r64["per_ms"], 99), "iters_mean": statistics.mean(iters64),
                 "setups_in_timed_region": sum(s["setup_called"] for s in r64["stats"])},
        "fp32_over_fp64": value / v64,
        "vcycle_gbs": {"fp32": f32.get("vcycle", {}).get("gbs"), "fp64": f64.get("vcycle", {}).get("gbs"),
                       "frac_fp32": (f32.get("vcycle", {}).get("gbs") or 0) / hbm,
                       "frac_fp64": (f64.get("vcycle", {}).get("gbs") or 0) / hbm},
        "vcycle_parts_us": {"note": "each part captured 20x into its own CUDA graph, device time per repetition",
                            "fp32": r32["parts"], "fp64": r64["parts"]},
        "families": {"fp32": f32, "fp64": f64,
                     "note": "CUDA-event brackets per family, from a separate timed region of "
                             f"{r32['profiled_steps']} steps per arm (bracketed step: "
                             f"{r32['profiled_ms_per_step']:.2f} ms fp32, {r64['profiled_ms_per_step']:.2f} ms fp64); "
                             "the level-0 sweeps (smooth0), nested in the V-cycle, in a further pass of their own"},
        "roofline": roof_family,
        "roofline_spmv": roof,
        "roofline_smoother_level0": roof_sm,
        "vcycle_hbm_frac_fp32": (f32.get("vcycle", {}).get("gbs") or 0) / hbm,
        "gpu_launches": int(r32["launches"]),
        "clocks": clocks,
    }
    if e2e is not None:
        line["e2e"] = e2e
    if batched is not None:
        line["batched"] = batched
    if serving is not None:
        line["serving"] = serving
    if natural is not None:
        line["bilu_natural"] = natural
    if numeric is not None:
        line["resetup_numeric"] = numeric
    if ua is not None:
        line["ua_amg"] = ua
    if alg45 is not None:
        line["alg45_coloring"] = alg45
    if adaptive is not None:
        line["adaptive_60x220x85"] = adaptive
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if err is not None:
        line["error_vs_oracle"] = err
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
