#!/usr/bin/env python
"""Benchmark: cell-steps/s of the full ADER-MOOD step (FP64) on the 3D bending column (a
1 x 1 x 6 box of 5,989,500 seeded tetrahedra, base clamped, lateral v = 0.1 (z/6)^2), the
largest single-mesh configuration; the 2D impact (999,698 triangles against a rigid slip wall)
is timed beside it, in an early window and in a mid-run window of its shock problem.

One step = one pass of the whole hot path: corner geometry, least-squares reconstruction,
ADER predictor and corner packets, nodal solver with BCs, forces and cell update, MOOD
detection and first-order recomputation, next dt. Inputs are resident in HBM before the
timed region; the working set (~5 GB for the column, ~0.5 GB for the impact) is larger than
L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload column3d|impact2d|cube3d]

Under torchrun (N > 1) every rank advances its own replica on its GPU (the path does not
shard across GPUs here); value = cell-steps of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-steps/s of full ADER-MOOD step (FP64, 1 GB300); batched and adjoint vs plain"
UNIT = "cell-steps/s"
WORKLOAD = "impact2d: 999,698 triangles (708x708 jittered Delaunay lattice), rho0=8.93 mu=0.46 lambda=1.06, v=(-0.1,0), slip wall x=0, CFL 0.4"
WORKLOADS = {
    "impact2d": WORKLOAD,
    "column3d": "column3d: 5,989,500 tetrahedra (55x55x330 jittered Kuhn cubes on 1x1x6), base clamped, rho0=1.1 mu=0.5 lambda=2.5, v=(0.1 (z/6)^2,0,0), CFL 0.25",
    "cube3d": "cube3d: 511,104 tetrahedra (44^3 jittered Kuhn cubes), slip walls, rho0=1 lambda=2, mu=1+0.2 GRF, Taylor-Green v0 (amplitude 0.05), CFL 0.25",
}


def make_workload(name: str):
    import workloads as W
    return {"impact2d": W.impact2d, "column3d": W.column3d, "cube3d": W.cube3d}[name]()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


# nominal GB300 FP64 rate: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz = 1.26 TFLOP/s
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def kernel_bytes(dim: int, nc: int, npn: int, nnz: int) -> dict:
    """Algorithmic (compulsory) DRAM bytes per full launch of each kernel class: every array
    the kernel needs is read once and every output written once (gathers of neighbours'
    data count once, as the data of the neighbour itself)."""
    D, NV = dim, dim + 1
    NS = D * (D + 1) // 2
    d8 = 8
    pk = d8 * (NS + D) * NV * nc
    # moments: node CSR, cells' x_c v F (once), x; writes the node moments
    nmom = 1 + D + NS + (D + D * D) * (1 + D)
    moments = 4 * (npn + 1) + 4 * NV * nc + d8 * (2 * D + D * D) * nc + d8 * D * npn + d8 * nmom * npn
    # predict: c2n, x, node moments, own x_c v F, mu z 1/m; writes packets and the order byte
    predict = (4 * NV * nc + d8 * D * npn + d8 * nmom * npn + d8 * (2 * D + D * D) * nc
               + 3 * d8 * nc + pk + nc)
    # nodes: CSR, packets, BC byte, x, v_p^n, rho (per cell, once); writes v*, x^{n+1},
    # v_p^{n+1} and the rho range per node
    nodes = (4 * (npn + 1) + 4 * NV * nc + pk + npn + 2 * d8 * D * npn + d8 * nc + 3 * d8 * D * npn
             + 2 * d8 * npn)
    # update: c2n, 5 node arrays + the node rho range, packets, v e F m 1/m mu, order;
    # writes v e F xc rho tau z, dt candidate
    update = (4 * NV * nc + 5 * d8 * D * npn + 2 * d8 * npn + pk + d8 * (D + 1 + D * D + 3) * nc + nc
              + d8 * (D + 1 + D * D + D + 3) * nc + d8 * nc)
    finalize = d8 * nc + 2 * nc
    return {"moments": moments, "predict": predict, "nodes": nodes, "update": update, "finalize": finalize}


# Per dimension, from one ncu capture of the current kernels (profiles/ holds its summary):
#  - FP64 floating-point operations per cell executed by each full-mesh kernel launch: ncu
#    counts of dadd + dmul + 2 dfma thread instructions divided by the cell count (they include
#    the FP64 expansions of division, sqrt, log, cbrt);
#  - FP64 thread instructions per cell (dfma + dadd + dmul): the pipe's issue rate, compared with
#    DGEMM's (one DFMA = 2 FLOP per instruction), shows how busy the pipe is independently of the
#    operation mix;
#  - DRAM bytes (read + write) per full launch per cell (the capture's traffic / its cells).
# COUNTS_SRC is the digest of the kernel sources the capture was taken on: when the sources
# differ the bench line says so ("counts_stale") and gives no traffic.
# 2D: impact2d (999,698 triangles), 3D: a reduced column (30 x 30 x 180 cubes, 972,000
# tetrahedra), both in profiles/column3d_kernels.md (the full meshes' traffic scales with the
# cells: every per-cell array is read and written once per launch).
FP64_FLOP_PER_CELL = {2: {"predict": 797.0, "update": 325.0, "nodes": 31.1, "moments": 120.0},
                      3: {"predict": 2333.0, "update": 688.0, "nodes": 48.5, "moments": 408.0}}
FP64_INSTR_PER_CELL = {2: {"predict": 481.0, "update": 210.0, "nodes": 25.0, "moments": 75.0},
                       3: {"predict": 1348.0, "update": 429.0, "nodes": 44.2, "moments": 240.0}}
TRAFFIC_PER_CELL = {2: {"predict": 373.2, "update": 464.5, "nodes": 181.6, "moments": 150.4},
                    3: {"predict": 643.0, "update": 860.1, "nodes": 413.0, "moments": 198.3}}
COUNTS_SRC = {2: "e26cc0dd37eaaecf", 3: "e26cc0dd37eaaecf"}
KERNEL_SOURCES = ("lmood_kernels.cuh", "lmood_dev.cuh", "lmood_ops_impl.cuh")


def kernel_source_digest() -> str:
    """sha256 (first 16 hex digits) of the forward kernels' sources"""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2104_02139_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def fp64_peak_tflops(device) -> float:
    """Measured FP64 peak: cuBLAS DGEMM 4096^3, best of 3 (CUDA events)."""
    import torch
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device=device)
    b = torch.randn(n, n, dtype=torch.float64, device=device)
    best = float("inf")
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2 * n ** 3 / (best / 1e3) / 1e12


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(pb, budget_s: float = 10.0) -> dict:
    """The oracle as it stands on the host cores: the first steps of the same workload, as
    many as the budget is expected to hold from the mean step time so far (at least one;
    set-up excluded), and at most 3 on a 3D mesh: the column's next steps start MOOD cascades,
    whose every round the oracle recomputes over the whole mesh (minutes of host time)."""
    import oracle as O
    O.build()
    t0 = time.perf_counter()
    o = O.Oracle(pb)
    setup = time.perf_counter() - t0
    steps, t = 0, 0.0
    cap = 3 if pb.mesh.dim == 3 else 50
    while steps < 1 or (t + t / steps <= budget_s and steps < cap):
        s0 = time.perf_counter()
        o.step()
        t += time.perf_counter() - s0
        steps += 1
    return {"value": pb.mesh.n_cells * steps / t, "unit": UNIT, "cores": O.threads(), "kind": "oracle",
            "sample": f"first {steps} steps of the same workload ({pb.mesh.n_cells} cells), {t:.1f} s of "
                      f"stepping after {setup:.1f} s of set-up; cores = the oracle's OpenMP threads"}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 0, 1, None
    import torch
    import torch.distributed as dist
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    dist.init_process_group(backend=backend)
    rank, local = dist.get_rank(), int(os.environ.get("LOCAL_RANK", "0"))
    return rank, local, ws, dist


def max_over_ranks(x: float, dist) -> float:
    if dist is None:
        return x
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


def job_throughput(ws: int, cells: int, steps: int, ms_max: float) -> float:
    """whole-job cell-steps/s: every rank advances its own replica of `cells` cells `steps`
    times; the job takes as long as its slowest rank (ms_max, the max over ranks)"""
    return ws * cells * steps / (ms_max / 1e3)


def reference_steps(pb, steps: int, warmup: int) -> dict:
    """The oracle as it stands on the host cores over the run's own warm-up and timed steps,
    each a bounded sample of the workload: its first time step from the initial data, the
    state (x, v_p, v, e, F, dt) restored before every step. Consecutive steps are not taken:
    from the column's second step on MOOD cascades start, and the oracle recomputes the whole
    mesh for each of their rounds (minutes of host time per step)."""
    if steps < 1 or warmup < 0:
        raise ValueError("the reference arm needs --steps >= 1 and --warmup >= 0")
    import oracle as O
    O.build()
    t0 = time.perf_counter()
    o = O.Oracle(pb)
    s0 = o.state()
    dt0 = o.dt
    setup = time.perf_counter() - t0
    t, rounds, troubled = 0.0, 0, 0
    for i in range(warmup + steps):
        o.set_state(x=s0["x"], vp=s0["vp"], v=s0["v"], e=s0["e"], F=s0["F"], dt=dt0)
        a = time.perf_counter()
        o.step()
        b = time.perf_counter()
        if i >= warmup:
            t += b - a
            rounds += o.info.mood_iters
            troubled += o.info.n_troubled
    o.close()
    n = pb.mesh.n_cells
    return {"value": n * steps / t, "unit": UNIT, "cores": O.threads(), "kind": "oracle",
            "ms_per_step": 1e3 * t / steps,
            "sample": f"each of the {steps} timed steps (after {warmup} untimed) is the workload's first time "
                      f"step from its initial data ({n} cells), the state restored before each; {t:.1f} s of "
                      f"stepping after {setup:.1f} s of set-up, {rounds} MOOD rounds and {troubled} troubled "
                      f"cells in the timed steps; cores = the oracle's OpenMP threads"}


def run_reference(args, rank, ws, dist):
    if rank != 0:
        return
    pb = make_workload(args.workload)
    cb = reference_steps(pb, args.steps, args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": cb.pop("ms_per_step"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload], "cells": pb.mesh.n_cells},
            "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, local, ws, dist):
    import torch
    import paper_2104_02139_gb300 as L
    import workloads as W

    torch.cuda.set_device(local)
    if rank == 0:  # one rank compiles (in-tree output); the others find it up to date
        L.build()
    barrier(dist)
    L.build()
    pb = make_workload(args.workload)
    N = pb.mesh.n_cells
    stream = torch.cuda.Stream()
    sim = L.simulation(pb, stream=stream.cuda_stream, graph=0 if args.host_mode else 1)
    info = sim.mesh.info()
    for _ in range(args.warmup):
        sim.step()
    tuned = None if args.no_autotune else sim.autotune()
    sched = None if args.no_autotune or args.host_mode else sim.autotune_schedule()
    for _ in range(2):  # re-capture the step graphs with the chosen launch shapes
        sim.step()
    first_timed = sim.info.step
    sim.timing(True)
    clocks = Clocks(local)
    barrier(dist)
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    troubled = 0
    for _ in range(args.steps):
        troubled += sim.step().n_troubled
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    kt = sim.timing_read()
    sim.timing(False)
    ms_max = max_over_ranks(ms, dist)
    value = job_throughput(ws, N, args.steps, ms_max)

    # roofline of the dominant kernel class (full-mesh launches; MOOD rounds excluded). The
    # step is bound by the FP64 pipe: roofline = FP64 FLOP/s against the FP64 peak, with the
    # HBM figure beside it.
    peaks, how = _peaks()
    kb = kernel_bytes(pb.mesh.dim, N, info["n_nodes"], info["stencil_nnz"])
    dom = max(("moments", "predict", "nodes", "update"), key=lambda k: kt[k][0])
    dom_ms = kt[dom][0] / max(kt[dom][1], 1)
    gbs = kb[dom] / (dom_ms / 1e3) / 1e9
    fp64_meas = None if args.no_fp64_peak else fp64_peak_tflops(f"cuda:{local}")
    fp64_peak = FP64_PEAK_TFLOPS  # an ALU-bound path: the peak derived from unit counts and clock
    hbm = {"achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
           "algorithmic_bytes_per_launch": kb[dom], "peak_source": how}
    dim = pb.mesh.dim
    fpc = FP64_FLOP_PER_CELL[dim].get(dom)
    digest = kernel_source_digest()
    stale = COUNTS_SRC[dim] is not None and COUNTS_SRC[dim] != digest
    if fpc:
        tf = fpc * N / (dom_ms / 1e3) / 1e12
        tpc = TRAFFIC_PER_CELL[dim].get(dom)
        roof = {"bound": "alu", "kernel": dom, "achieved": tf, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": tf / fp64_peak, "traffic": None if (stale or tpc is None) else tpc * N,
                "peak_source": "derived: 152 SMs x 2 DFMA lanes/clk x 2 FLOP x 2.07 GHz max SM clock",
                "dgemm_measured": fp64_meas, "frac_of_dgemm": (tf / fp64_meas) if fp64_meas else None,
                "fp64_flop_per_cell": fpc, "ms_per_launch": dom_ms, "hbm": hbm,
                "counts_src": COUNTS_SRC[dim], "kernel_src": digest, "counts_stale": stale}
        ipc = FP64_INSTR_PER_CELL[dim].get(dom)
        if ipc:
            gi = ipc * N / (dom_ms / 1e3) / 1e9
            roof["fp64_issue"] = {"achieved": gi, "peak": fp64_peak * 1e3 / 2, "unit": "G FP64 instr/s",
                                  "frac": gi / (fp64_peak * 1e3 / 2), "fp64_instr_per_cell": ipc,
                                  "frac_of_dgemm": (gi / (fp64_meas * 1e3 / 2)) if fp64_meas else None}
    else:
        roof = {"bound": "hbm", "kernel": dom, "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": gbs / peaks["hbm_gbs"], "traffic": None, "peak_source": how,
                "algorithmic_bytes_per_launch": kb[dom], "ms_per_launch": dom_ms, "fp64_peak_measured": fp64_meas}
    kernels = {k: {"ms_total": v[0], "launches": v[1]} for k, v in kt.items()}
    launches = sum(v[1] for v in kt.values())

    # end to end through the C ABI with host buffers: every step uploads the state from
    # pinned host memory, steps, and reads the new state back
    e2e = None
    if not args.no_e2e:
        d = pb.mesh.dim
        fields = ((L.FIELD_X, (d, info["n_nodes"])), (L.FIELD_VP, (d, info["n_nodes"])), (L.FIELD_V, (d, N)),
                  (L.FIELD_E, (N,)), (L.FIELD_F, (d * d, N)), (L.FIELD_DT, (1,)))
        bufs = {f: torch.empty(shp, dtype=torch.float64, pin_memory=True).numpy() for f, shp in fields}
        for f, _ in fields:
            sim.get(f, out=bufs[f])
        nbytes = sum(b.nbytes for b in bufs.values())
        k2 = max(5, args.steps // 4)
        torch.cuda.synchronize()
        part = [0.0, 0.0, 0.0]  # host wall time of the set (H2D + refresh), the step, the get (D2H)
        t0 = time.perf_counter()
        for _ in range(k2):
            ta = time.perf_counter()
            sim.set_fields(bufs)
            tb = time.perf_counter()
            sim.step()
            tc = time.perf_counter()
            sim.get_fields(bufs)
            td = time.perf_counter()
            part[0] += tb - ta
            part[1] += tc - tb
            part[2] += td - tc
        torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - t0, dist)
        e2e = {"value": ws * N * k2 / el, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "steps": k2,
               "ms_per_step": {"set_h2d": 1e3 * part[0] / k2, "step": 1e3 * part[1] / k2, "get_d2h": 1e3 * part[2] / k2},
               "gb_per_s": {"h2d": nbytes * k2 / part[0] / 1e9, "d2h": nbytes * k2 / part[2] / 1e9}}

    impact = None
    if not args.no_impact and args.workload != "impact2d":
        sim.close()
        sim.mesh.close()
        impact = run_impact_windows(L, W, torch, args)

    batched = None
    if not args.no_batched:
        # the batch is 2D: its ratio is taken to the plain 2D step (the impact's early window)
        plain2d = impact["early"]["value"] if impact else (value / ws if pb.mesh.dim == 2 else None)
        batched = run_batched(L, W, torch, local, plain2d, args)

    variants = None
    if not args.no_variants:
        variants = run_variants(L, W, torch, pb, value / ws, args)

    adjoint = None
    if not args.no_adjoint:
        sim.close()
        sim.mesh.close()
        adjoint = run_adjoint(L, W, torch, args)

    cb = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(pb)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOADS[args.workload], "cells": N, "nodes": info["n_nodes"],
                           "lsq_pairs": info["stencil_nnz"], "parallelism": f"replicas x{ws}",
                           "l2": "working set > L2 (no flush)", "troubled_cells_in_timed_steps": troubled,
                           "troubled_frac": troubled / (N * args.steps), "first_timed_step": first_timed},
                "roofline": roof, "kernels": kernels, "gpu_launches": launches, "clocks": ck, "e2e": e2e,
                "cpu_baseline": cb, "impact2d_windows": impact, "batched": batched, "variants": variants,
                "adjoint": adjoint,
                "launch": None if tuned is None else {**{k: v["chosen"] for k, v in tuned.items()},
                                                      **({} if sched is None else
                                                         {"node_window": sched["node_window"]["chosen"],
                                                          "step_form": sched["step_form"]["chosen"],
                                                          "step_form_ms": sched["step_form"]["ms"],
                                                          "node_window_ms": sched["node_window"]["ms"]})}}
        print(json.dumps(line), flush=True)


def _timed_window(sim, N, k, stream, torch) -> dict:
    """k graph-captured steps of sim under CUDA events (per-stage timing on): cell-steps/s, the
    troubled and first-order fractions, MOOD rounds and MOOD loop time per step."""
    sim.timing(True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    tr = p0 = it = 0
    for _ in range(k):
        info = sim.step()
        tr += info.n_troubled
        p0 += info.n_p0
        it += info.mood_iters
    e1.record(stream)
    torch.cuda.synchronize()
    kt = sim.timing_read()
    sim.timing(False)
    ms = e0.elapsed_time(e1) / k
    stage_ms = sum(v[0] for v in kt.values())
    mood_ms = kt["mood"][0] / k
    return {"steps": k, "ms_per_step": ms, "value": N / (ms / 1e3), "unit": UNIT,
            "troubled_frac": tr / (N * k), "p0_frac": p0 / (N * k), "mood_rounds_per_step": it / k,
            "mood_ms_per_step": mood_ms, "mood_share": kt["mood"][0] / stage_ms if stage_ms > 0 else None,
            "mood_us_per_round": 1e3 * mood_ms / (it / k) if it else None,
            "mood_ns_per_troubled_cell": 1e6 * mood_ms / (tr / k) if tr else None,
            "t": float(sim.info.t)}


def run_impact_windows(L, W, torch, args) -> dict:
    """The 2D impact (999,698 triangles, the shock problem of the configurations) in two timed
    windows of K graph-captured steps each: early (from step 8, as the front forms) and mid-run
    (from step args.midrun_from, with the compression front and its troubled band established).
    Per window: cell-steps/s, the troubled fraction (cells sent down the cascade per cell-step),
    the first-order fraction, MOOD rounds per step and the MOOD loop's share of the step time
    (CUDA events around each stage). Then the MOOD load curve: the early window again with the
    RDMP relaxations delta0, delta1 scaled by 0.1, 0.01 and 0 (a stricter detection, so that
    more cells go down the cascade: the cost of the MOOD loop against the troubled fraction),
    and the same impact on a 19,602-triangle mesh, where the troubled band is a few percent
    of the cells as on the paper's meshes."""
    pb = W.impact2d()
    N = pb.mesh.n_cells
    stream = torch.cuda.Stream()
    graph = 0 if args.host_mode else 1
    sim = L.simulation(pb, stream=stream.cuda_stream, graph=graph)
    k = max(10, args.steps)
    out, taken = {}, 0
    for name, first in (("early", 8), ("mid_run", args.midrun_from)):
        while taken < first:
            sim.step()
            taken += 1
        out[name] = {"first_step": first, **_timed_window(sim, N, k, stream, torch)}
        taken += k
    sim.close()
    sim.mesh.close()
    d0 = L.params_default(2)
    load = []
    for scale in (0.1, 0.01, 0.0):
        sim = L.simulation(pb, stream=stream.cuda_stream, graph=graph, delta0=d0.delta0 * scale,
                           delta1=d0.delta1 * scale)
        try:
            for _ in range(8):
                sim.step()
            load.append({"delta_scale": scale, "first_step": 8, **_timed_window(sim, N, k, stream, torch)})
        except L.LmoodError as e:  # a status of the library (e.g. the MOOD round limit), not a crash
            load.append({"delta_scale": scale, "error": str(e)})
        sim.close()
        sim.mesh.close()
    # the same impact at a resolution like the paper's meshes (100 x 100 points, 19,602
    # triangles): the front's band of cells is then a few percent of the mesh
    pbs = W.impact2d(n=100)
    sim = L.simulation(pbs, stream=stream.cuda_stream, graph=graph)
    try:
        for _ in range(8):
            sim.step()
        load.append({"delta_scale": 1.0, "cells": pbs.mesh.n_cells, "first_step": 8,
                     **_timed_window(sim, pbs.mesh.n_cells, k, stream, torch)})
    except L.LmoodError as e:
        load.append({"delta_scale": 1.0, "cells": pbs.mesh.n_cells, "error": str(e)})
    sim.close()
    sim.mesh.close()
    out["mood_load"] = load
    out["cells"] = N
    out["what"] = ("impact2d in two windows of its run: troubled_frac = cells sent down the cascade per "
                   "cell-step (the paper's 'troubled cells per step'), mood_share = MOOD loop time / step time; "
                   "mood_load: the early window with delta0, delta1 scaled down (stricter RDMP)")
    return out


def run_variants(L, W, torch, pb, plain_value, args) -> dict:
    """The scheme's variants, each timed like the plain step (graph-captured steps, CUDA events,
    after 5 untimed steps): on the benchmark mesh the shear energy family with a = 0 and the
    three-level cascade (P1 -> P1 with Barth-Jespersen slopes -> P0); on 316 x 316-point
    unit squares (198,450 triangles) a piston (prescribed-velocity face, slip walls) and a block
    pressed against a contact wall (0.7 h away at the start); on 44^3 Kuhn cubes (511,104 tets) the stiffened-gas jelly
    block dropped on a contact floor; the 40 x 40-point unit square (3,042 triangles) with
    graph-captured steps and with the persistent step (one cooperative launch per step).
    cell-steps/s, and for the first two the ratio to the plain step on the same mesh."""
    import dataclasses
    cases = [("shear_family_a0", dataclasses.replace(pb, shear_a=0.0), {}, True),
             ("cascade3_bj", pb, {"cascade": 3}, True),
             ("piston_velocity_faces", W.piston2d(n=316), {}, False),
             ("contact_rebound", W.rebound2d(n=316, gap=0.7 / 315), {}, False),  # in contact after ~5 steps
             ("stiffened_gas_jelly_drop_3d", W.jellydrop3d(n=44), {}, False)]
    small = W.plain2d(n=40)  # 3,042 triangles: latency-bound
    cases += [("small_plain2d_graph", small, {}, False), ("small_plain2d_persistent", small, {"graph": 2}, False)]
    out = {}
    stream = torch.cuda.Stream()
    for name, q, kw, same_mesh in cases:
        kw = {"graph": 0 if args.host_mode else 1, **kw}
        sim = L.simulation(q, stream=stream.cuda_stream, **kw)
        for _ in range(5):
            sim.step()
        k = 40
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        troubled = 0
        for _ in range(k):
            troubled += sim.step().n_troubled
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k
        v = q.mesh.n_cells / (ms / 1e3)
        out[name] = {"cells": q.mesh.n_cells, "ms_per_step": ms, "value": v, "unit": UNIT, "steps": k,
                     "troubled_cells": troubled}
        if same_mesh:
            out[name]["vs_plain"] = v / plain_value
        sim.close()
        sim.mesh.close()
    # the 40 x 40 configuration (3,042 triangles) as configured: 200 steps in one lmood_run,
    # chained on the device (one host synchronisation for the run)
    sim = L.simulation(small, stream=stream.cuda_stream)
    sim.run(5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = sim.run(200)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    out["small_plain2d_run200_chained"] = {"cells": small.mesh.n_cells, "ms_per_step": el * 1e3 / 200,
                                           "us_per_step": el * 1e6 / 200, "value": small.mesh.n_cells * 200 / el,
                                           "unit": UNIT, "steps": 200, "host_syncs": info.syncs,
                                           "timer": "host wall clock around lmood_run (includes its one sync)"}
    sim.close()
    sim.mesh.close()
    return out


def run_batched(L, W, torch, local, plain_value, args) -> dict:
    """Batched configuration: 256 independent unit-square meshes (sizes log-uniform in [1e3, 2e5]
    cells, own mu, amplitude and dt each) concatenated and advanced by one launch per stage in
    graph-captured steps; cell-steps/s over all instances, and the ratio to the plain step."""
    t0 = time.perf_counter()
    probs = W.batched2d(workers=min(16, os.cpu_count() or 1))
    pb, inst = W.concat(probs)
    gen = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    sim = L.simulation(pb, stream=stream.cuda_stream, cell_inst=inst, n_inst=len(probs),
                       graph=0 if args.host_mode else 1)
    for _ in range(3):
        sim.step()
    tuned = None
    if not args.no_autotune:
        blocks = sim.autotune()
        sched = sim.autotune_schedule()
        tuned = {"blocks": {k2: v["chosen"] for k2, v in blocks.items()},
                 "node_window": sched["node_window"]["chosen"], "step_form": sched["step_form"]["chosen"],
                 "step_form_ms": sched["step_form"]["ms"]}
        sim.step()
    k = max(10, args.steps // 5)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    tr = 0
    for _ in range(k):
        tr += sim.step().n_troubled
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    val = pb.mesh.n_cells * k / (ms / 1e3)
    dt = sim.get(L.FIELD_DT)
    return {"value": val, "unit": UNIT, "vs_plain_2d": val / plain_value if plain_value else None,
            "plain_2d_value": plain_value, "instances": len(probs),
            "cells": pb.mesh.n_cells, "steps": k, "ms_per_step": ms / k, "troubled_cells": tr,
            "dt_min": float(dt.min()), "dt_max": float(dt.max()), "mesh_generation_s": gen,
            "launch": "one launch per stage for all instances, graph-captured steps", "autotuned": tuned}


def run_adjoint(L, W, torch, args) -> dict:
    """Adjoint configuration (511,104-tet cube, per-cell mu from a Gaussian random field,
    Taylor-Green v0): gradient of J = sum over cells with initial centroid z > 0.5 of
    m |v|^2 / 2 after K steps with respect to the initial v0 and mu (through the initial
    nodal solve), MOOD masks and dt frozen at their recorded values. Times: the plain step of
    the same configuration, the recording (the K ordinary steps plus what the tape keeps), and
    the reverse pass, per step; store mode (every state and step product kept) and
    checkpoints every 20 steps with recomputation."""
    pb = W.cube3d()
    d, nc = pb.mesh.dim, pb.mesh.n_cells
    zc = pb.mesh.x[2][pb.mesh.c2n].mean(axis=0)
    sel = torch.tensor(zc > 0.5, device="cuda")
    stream = torch.cuda.Stream()
    kf, runs = 50, []
    for _ in range(2):  # the same 50 steps from two fresh states: the faster run (host jitter
        # between the synchronised steps shows up as device idle time)
        fw = L.simulation(pb, stream=stream.cuda_stream, graph=0 if args.host_mode else 1)
        for _ in range(3):
            fw.step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(kf):
            fw.step()
        e1.record(stream)
        torch.cuda.synchronize()
        runs.append(e0.elapsed_time(e1) / kf)
        fw.close()
        fw.mesh.close()
    fwd_ms = min(runs)
    k = args.adjoint_steps
    res = {"steps": k, "cells": nc, "forward_ms_per_step": fwd_ms, "forward_ms_runs": runs,
           "forward_cell_steps_per_s": nc / (fwd_ms / 1e3)}
    for ck in (0, 20):
        sim = L.simulation(pb, stream=stream.cuda_stream, graph=0 if args.host_mode else 1)
        m = torch.empty(nc, dtype=torch.float64, device="cuda")
        v = torch.empty((d, nc), dtype=torch.float64, device="cuda")
        out = {key: torch.empty(shp, device="cuda", dtype=torch.float64)
               for key, shp in (("v", (d, nc)), ("mu", (nc,)))}
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        try:
            tape = L.Tape(sim, k, ck)
        except L.LmoodError as err:
            if err.status != L.ERR_OOM:
                raise
            res[f"checkpoint_every_{ck}"] = {"skipped": "device memory"}
            sim.close()
            continue
        e1.record(stream)
        sim.get(L.FIELD_MASS, m)
        sim.get(L.FIELD_V, v)
        with torch.cuda.stream(stream):
            lam_v = torch.where(sel, m, torch.zeros_like(m)) * v  # dJ/dv^N
            J = float((0.5 * torch.where(sel, m, torch.zeros_like(m)) * (v * v).sum(0)).sum())
        torch.cuda.synchronize()  # the objective's torch ops are not part of the reverse pass
        e3 = torch.cuda.Event(enable_timing=True)
        e3.record(stream)
        tape.backward(lam_v=lam_v, out=out)
        e2.record(stream)
        torch.cuda.synchronize()
        rec, bwd = e0.elapsed_time(e1) / k, e3.elapsed_time(e2) / k
        res[f"checkpoint_every_{ck}"] = {"record_ms_per_step": rec, "backward_ms_per_step": bwd,
                                         "backward_over_forward": bwd / fwd_ms,
                                         "record_over_forward": rec / fwd_ms, "tape_bytes": tape.info()["bytes"],
                                         "J": J, "grad_v0_norm": float(out["v"].norm()),
                                         "grad_mu_norm": float(out["mu"].norm())}
        tape.close()
        sim.close()
        sim.mesh.close()
    res["what"] = ("J = sum_{z_c(0) > 0.5} m |v|^2 / 2 at t^K; gradient w.r.t. v0 and mu per cell "
                   "(through the initial nodal solve); MOOD masks and dt frozen")
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="column3d",
                    help="column3d (the largest single-mesh configuration, default), impact2d or cube3d")
    ap.add_argument("--no-impact", action="store_true", help="skip the impact2d early / mid-run windows")
    ap.add_argument("--midrun-from", type=int, default=400, help="first step of the impact2d mid-run window")
    ap.add_argument("--host-mode", action="store_true",
                    help="host-driven MOOD rounds instead of graph-captured steps (same kernels; for profilers)")
    ap.add_argument("--no-fp64-peak", action="store_true", help="skip the DGEMM FP64 peak measurement")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-instances measurement")
    ap.add_argument("--no-variants", action="store_true", help="skip the boundary / material / cascade variants")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the reverse-pass measurement")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--adjoint-steps", type=int, default=400, help="steps recorded for the adjoint measurement")
    ap.add_argument("--case", type=int, default=0,
                    help="profiling case: build the workload, take this many untimed steps, exit")
    ap.add_argument("--case-adjoint", type=int, default=0,
                    help="with --case: then record this many steps on a tape and run its reverse pass once")
    ap.add_argument("--case-n", type=int, default=0,
                    help="with --case: a smaller impact2d (lattice n x n), cube3d (n^3 cubes) or column3d "
                         "(n x n x 6n cubes) for multi-pass profiler captures")
    ap.add_argument("--case-ckpt", type=int, default=0,
                    help="with --case-adjoint: the tape's checkpoint interval (0: store mode)")
    args = ap.parse_args()
    if args.case:
        import torch
        import paper_2104_02139_gb300 as L
        import workloads as W
        L.build()
        if args.case_n:
            if args.workload == "column3d":
                pb = W.column3d(nxy=args.case_n, nz=6 * args.case_n)
            else:
                pb = {"impact2d": W.impact2d, "cube3d": W.cube3d}[args.workload](n=args.case_n)
        else:
            pb = make_workload(args.workload)
        sim = L.simulation(pb, graph=0 if args.host_mode else 1)
        for _ in range(args.case):
            info = sim.step()
        if args.case_adjoint:
            tape = L.Tape(sim, args.case_adjoint, args.case_ckpt)
            g = tape.backward(lam_v=np.ones(sim.shape(L.FIELD_V)))
            print(f"case adjoint: {args.case_adjoint} steps, |grad v| max {np.abs(g['v']).max():.6g}")
        torch.cuda.synchronize()
        print(f"case: {args.case} steps, last dt {info.dt_used:.6g}, troubled {info.n_troubled}")
        return
    rank, local, ws, dist = dist_setup()
    try:
        if args.impl == "reference":
            run_reference(args, rank, ws, dist)
        else:
            run_ours(args, rank, local, ws, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
