#!/usr/bin/env python
"""Throughput of the MHD step on GB300: zone-updates/s on the 256^3 turbulent box.

Workload: 3D periodic driven-free turbulence, 256^3 cells, gamma = 5/3, rho = 1, p = 1,
B = (0.1, 0, 0), seeded solenoidal velocity (2 <= |k| <= 8, shell spectrum ~ k^-2,
rms Mach 2), CFL 0.4 with the time step computed on the device every step.  A step
is one full van Leer predictor-corrector step (recovery, HLLD fluxes in x/y/z,
corner EMFs, update of cells and faces, CFL reduction) of the mixed path (FP32 bulk,
FP64 pressure recovery and state accumulation), replayed from a captured CUDA graph.
The plain FP64 path is timed on the same box and reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun): every rank advances its own box (independent replicas, seed offset
by rank): weak scaling, no data-path collective; timing uses a barrier and the max
over ranks.  --impl reference times the FP64 CPU oracle of the same step on the
host cores (a bounded sample of the workload).
"""
from __future__ import annotations

import argparse
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

N_CELLS = 256
CFL = 0.4
SEED = 1502
# measured peaks (driver-written) with the recipe's fallback
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
SM_COUNT = 152
FP32_LANES_PER_SM = 128

# algorithmic work per item of each kernel class ("Roofline"):
#   flops  : FP32 (mixed) arithmetic of the method per item, FMA counted as 2
#   bytes  : unique HBM bytes per item (mixed path, FP32 scratch)
KCLASS = {
    "recovery": dict(bound="hbm", flops=60, bytes=64 + 8 * 4, unit="padded cell"),
    "flux1_x": dict(bound="alu", flops=343, bytes=7 * 4 + 8 + 7 * 4, unit="face"),
    "flux1_y": dict(bound="alu", flops=343, bytes=7 * 4 + 8 + 7 * 4, unit="face"),
    "flux1_z": dict(bound="alu", flops=343, bytes=7 * 4 + 8 + 7 * 4, unit="face"),
    "flux2_x": dict(bound="alu", flops=553, bytes=7 * 4 + 8 + 7 * 4, unit="face"),
    "flux2_y": dict(bound="alu", flops=553, bytes=7 * 4 + 8 + 7 * 4, unit="face"),
    "flux2_z": dict(bound="alu", flops=553, bytes=7 * 4 + 8 + 7 * 4, unit="face"),
    "emf": dict(bound="hbm", flops=75, bytes=(9 + 6 + 3) * 4, unit="edge point"),
    "update": dict(bound="hbm", flops=50, bytes=18 * 4 + 64 + 16 + 64, unit="cell"),
}


def units_per_launch(cls: str, n: int) -> int:
    if cls == "recovery":
        return (n + 4) ** 3
    if cls.startswith("flux"):
        return (n + 1) * (n + 2) * (n + 2)
    return (n + 1) ** 3


def load_peaks():
    try:
        with open(PEAKS_PATH) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), float(pk.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


# ---------------------------------------------------------------- clocks ----
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-i", str(self.device), "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ distributed ----
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, v: float) -> float:
    if pg is None:
        return v
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# -------------------------------------------------------------- CPU oracle ----
def oracle_sample(target_s: float = 15.0, n: int = 64, max_steps: int = 50):
    """Time the FP64 CPU oracle on an n^3 box of the same recipe, all host cores."""
    import oracle
    from paper_1502_02935_gb300 import inputs
    cores = oracle.set_threads(os.cpu_count() or 1)
    st = inputs.turbulence(n, seed=SEED)
    steps, t0 = 0, time.perf_counter()
    while steps < max_steps:
        dt = oracle.cfl_dt(st, CFL)
        st = oracle.step(st, dt)
        steps += 1
        if time.perf_counter() - t0 > target_s:
            break
    el = time.perf_counter() - t0
    return {"value": n ** 3 * steps / el, "unit": "zone-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"{n}^3 box of the same turbulence recipe (seed {SEED}), {steps} CFL steps, "
                      f"{el:.1f} s wall on {cores} host threads (FP64, plain C, OpenMP)"}


def run_reference(args, world, rank, pg):
    if rank != 0:
        return 0
    cb = oracle_sample(target_s=max(5.0, min(60.0, 2.0 * args.steps)))
    line = {"impl": "reference", "metric": "zone-updates/s", "value": cb["value"], "unit": "zone-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "turbulence_256^3 (oracle timed on a 64^3 sample of the same recipe)",
                       "global_batch": 1, "seq_len": 0, "parallelism": "replicas"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "zone-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- GPU path ----
def timed_steps(grid, steps: int, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        grid.step(-1.0)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def run_ours(args, world, rank, local, pg):
    import torch
    from paper_1502_02935_gb300 import inputs, mhd

    torch.cuda.set_device(local)
    hbm_peak, sm_max_mhz, peak_kind = load_peaks()
    n = args.n
    zones = n ** 3
    st = inputs.turbulence(n, seed=SEED + rank)
    stream = torch.cuda.Stream()
    grid = mhd.Grid(st, precision="mixed", cfl=CFL, flags=mhd.FLAG_GRAPH, stream=stream.cuda_stream)
    for _ in range(args.warmup):
        grid.step(-1.0)
    torch.cuda.synchronize()
    barrier(pg)
    torch.cuda.synchronize()
    l0 = grid.launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    ms = timed_steps(grid, args.steps, stream)
    clk = clocks.stop()
    torch.cuda.synchronize()
    barrier(pg)
    launches = grid.launch_count() - l0
    ms = max_over_ranks(pg, ms)
    value = zones * args.steps * world / (ms / 1e3)
    grid.sync()

    # per-kernel times of the same step sequence (events on the library's stream)
    grid.set_profiling(True)
    kp = max(3, min(args.steps, 10))
    for _ in range(kp):
        grid.step(-1.0)
    prof = grid.profile()
    grid.set_profiling(False)
    tot = sum(v[0] for v in prof.values()) or 1.0
    dom = max((k for k in prof if k in KCLASS), key=lambda k: prof[k][0])
    dom_ms = prof[dom][0] / max(prof[dom][1], 1)
    kc = KCLASS[dom]
    units = units_per_launch(dom, n)
    clk_mhz = (clk or {}).get("sm_mhz") or sm_max_mhz
    if kc["bound"] == "alu":
        peak = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
        achieved = kc["flops"] * units / (dom_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": dom,
                "peak_note": f"FP32 FMA peak 152 SMs x 128 lanes x 2 x {sm_max_mhz:.0f} MHz (derived)"}
    else:
        achieved = kc["bytes"] * units / (dom_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None, "kernel": dom, "peak_note": f"{peak_kind} hbm_gbs"}
    shares = {k: round(v[0] / tot, 4) for k, v in prof.items() if v[1]}

    # plain FP64 path on the same box
    g64 = mhd.Grid(st, precision="fp64", cfl=CFL, flags=mhd.FLAG_GRAPH, stream=stream.cuda_stream)
    g64.step(-1.0)
    torch.cuda.synchronize()
    k64 = max(2, min(args.steps, 6))
    ms64 = timed_steps(g64, k64, stream)
    ms64 = max_over_ranks(pg, ms64)
    fp64_value = zones * k64 * world / (ms64 / 1e3)
    g64.close()

    # end to end through the C ABI with host buffers: H2D of the step's input and D2H of
    # its result inside the timed region
    U_h = torch.from_numpy(np.ascontiguousarray(st.U)).pin_memory()
    B_h = torch.from_numpy(np.ascontiguousarray(st.faces_flat())).pin_memory()
    ke = max(2, min(args.steps, 5))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(ke):
        grid.set_state_ptr(0, U_h.data_ptr(), B_h.data_ptr(), False)
        grid.step(-1.0)
        grid.get_state_ptr(0, U_h.data_ptr(), B_h.data_ptr(), False)
    e1.record(stream)
    e1.synchronize()
    ms_e2e = max_over_ranks(pg, e0.elapsed_time(e1))
    e2e_value = zones * ke * world / (ms_e2e / 1e3)
    io_bytes = (U_h.numel() + B_h.numel()) * 8
    grid.close()

    if rank != 0:
        return 0
    cb = oracle_sample(target_s=15.0) if world == 1 or rank == 0 else None
    line = {
        "metric": "zone-updates/s", "value": value, "unit": "zone-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded solenoidal turbulence, no dataset)",
        "config": {"workload": f"turbulence_{n}^3 periodic MHD, gamma=5/3, B=(0.1,0,0), rms Mach 2, CFL {CFL}, "
                               "mixed precision (FP32 bulk, FP64 recovery+accumulation), graph replay",
                   "cells": zones, "global_batch": world, "seq_len": 0,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (state 1.1 GB/replica, no flush)"},
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": "zone-updates/s", "h2d_bytes_per_step": io_bytes,
                "d2h_bytes_per_step": io_bytes},
        "gpu_launches": launches,
        "roofline": roof,
        "hbm_alg_frac": value / world * 128.0 / (hbm_peak * 1e9),
        "fp64_path": {"value": fp64_value, "unit": "zone-updates/s", "steps": k64},
        "kernel_shares": shares,
        "cpu_baseline": cb,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_CELLS, help="cells per axis (default 256)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local, pg = dist_setup()
    try:
        if args.impl == "reference":
            return run_reference(args, world, rank, pg)
        return run_ours(args, world, rank, local, pg)
    finally:
        if pg is not None:
            pg.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
