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
import datetime
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
REF_SAMPLE_N = 64  # edge of the box the oracle arm times (the full box takes minutes per step)
CFL = 0.4
SEED = 1502
# measured peaks (driver-written) with the recipe's fallback
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
SM_COUNT = 152
FP32_LANES_PER_SM = 128

# Algorithmic work per item of each kernel class of the mixed path, counted from the
# formulas the kernels evaluate: FP64 pipe operations of the precision split (an add, a
# multiply or an FMA is one operation: each holds the FP64 pipe for the same time), FP32
# flops of the bulk arithmetic (FMA = 2), and unique HBM bytes.  A kernel's roofline is the
# resource it uses the largest fraction of.
KCLASS = {
    # recovery: three face sums, |m|^2 and |B|^2 (3 + 3), Newton step of 1/rho (2), p (4)
    "recovery": dict(fp64=15, fp32=30, bytes=64 + 8 * 4, unit="padded cell"),
    "flux1_x": dict(fp64=0, fp32=343, bytes=7 * 4 + 8 + 7 * 4, unit="face"),
    "flux1_y": dict(fp64=0, fp32=343, bytes=7 * 4 + 8 + 7 * 4, unit="face"),
    "flux1_z": dict(fp64=0, fp32=343, bytes=7 * 4 + 8 + 7 * 4, unit="face"),
    # the three donor-cell directions in one kernel (three active axes): per face
    "flux1_xyz": dict(fp64=0, fp32=343, bytes=7 * 4 + 8 + 7 * 4, unit="face"),
    "flux2_x": dict(fp64=0, fp32=553, bytes=7 * 4 + 8 + 7 * 4, unit="face"),
    "flux2_y": dict(fp64=0, fp32=553, bytes=7 * 4 + 8 + 7 * 4, unit="face"),
    "flux2_z": dict(fp64=0, fp32=553, bytes=7 * 4 + 8 + 7 * 4, unit="face"),
    "emf": dict(fp64=0, fp32=60, bytes=(8 + 3 + 3) * 4, unit="edge point"),
    # update fused with the recovery of the new state: FP64 = 14 adds (cell, six faces, three
    # face sums) + |m|^2 and |B|^2 (3 + 3) + Newton step of 1/rho (2) + p (4); bytes = F (60) +
    # E (12) + base U (64) + new U (64) + new W and cell EMF (44)
    "update": dict(fp64=26, fp32=140, bytes=15 * 4 + 3 * 4 + 64 + 64 + 11 * 4, unit="point"),
    "ghost": dict(fp64=0, fp32=0, bytes=11 * 4 * 2, unit="ghost point"),
    # corner EMFs fused with the update (three active axes): FP64 = 5 cell adds + 3 face
    # updates + 3 face sums + 12 recovery; bytes = F of three directions (84) + cell EMFs of
    # the input state (12) + base U (64) + new U (64; the predictor of a periodic box without
    # potential stores its 24 B of faces only) + new W and cell EMF (44)
    "emf_update": dict(fp64=23, fp32=200, bytes=21 * 4 + 3 * 4 + 64 + (64 + 24) / 2 + 11 * 4, unit="cell"),
}
# FP64 pipe operations per clock per SM: the nominal 1.25 TFLOP/s of the part is
# 152 SMs x 2 FMAs x 2 flops x ~2.06 GHz.  (A DFMA probe measured 1.0 TFLOP/s.)
FP64_OPS_PER_SM_CLK = 2
# The step's algorithmic HBM bytes per cell: read the 8 FP64 fields of U^n, write U^n+1.
ALG_BYTES_PER_CELL = 128.0
# DRAM bytes (read + write) per item of the dominant kernel, from one ncu capture of each
# stage of the EMF + update kernel on turbulence 192^3 (corrector 2.037 GB, predictor 1.734 GB
# per launch over 192^3 cells, ten planes per CTA as on 256^3), their mean scaled by the items
# of a launch.  Retake it when the kernel changes.
MEASURED_DRAM_BYTES_PER_POINT = {"emf_update": 0.5 * (2.037e9 + 1.734e9) / 192 ** 3}
MEASURED_DRAM_NOTE = {"emf_update": "ncu dram bytes (read + write) at turbulence 192^3, mean of the predictor "
                                    "and corrector launches, per cell, scaled to this launch"}


def units_per_launch(cls: str, n: int) -> int:
    if cls == "recovery":
        return (n + 4) ** 3
    if cls == "ghost":
        return (n + 4) ** 3 - n ** 3
    if cls == "flux1_xyz":
        return 3 * (n + 1) * (n + 2) * (n + 2)
    if cls.startswith("flux"):
        return (n + 1) * (n + 2) * (n + 2)
    if cls == "emf_update":
        return n ** 3
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
    """nvidia-smi every 50 ms into a file; `stop(t0, t1)` keeps the samples whose timestamps
    fall inside the timed window [t0, t1] (host wall clock), else the one nearest to it."""
    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
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
                                          "-i", str(self.device), "-lms", "50"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def wait_first(self, timeout: float = 3.0):
        """Block until nvidia-smi has written its first line (its start-up takes a while)."""
        t = time.time()
        while self.proc is not None and time.time() - t < timeout:
            self.fh.flush()
            if os.path.getsize(self.path) > 0:
                return
            time.sleep(0.02)

    def stop(self, t0: float, t1: float):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        inside = [r for r in rows if t0 <= r[0] <= t1]
        if not inside:
            inside = [min(rows, key=lambda r: min(abs(r[0] - t0), abs(r[0] - t1)))]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = {nm for r in inside for nm, v in zip(names, r[3]) if v.lower() in ("active", "1")}
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": inside[0][2],
                "reasons": sorted(reasons), "samples": len(inside),
                "in_window": t0 <= inside[0][0] <= t1}


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


def workload_config(n: int, world: int) -> dict:
    """The workload both arms report: the problem, its size and the parallel layout."""
    return {"workload": f"turbulence_{n}^3 periodic MHD, gamma=5/3, B=(0.1,0,0), rms Mach 2, CFL {CFL}",
            "cells": n ** 3, "global_batch": world, "seq_len": 0,
            "parallelism": "replicas" if world > 1 else "single"}


def run_reference(args, world, rank, pg):
    if rank != 0:
        return 0
    cb = oracle_sample(target_s=max(5.0, min(60.0, 2.0 * args.steps)), n=REF_SAMPLE_N)
    line = {"impl": "reference", "metric": "zone-updates/s", "value": cb["value"], "unit": "zone-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(REF_SAMPLE_N, args.gpus),
                           sample=f"the FP64 oracle timed on a {REF_SAMPLE_N}^3 box of the {args.n}^3 workload's "
                                  f"recipe, on the host cores"),
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


def run_batched(args, stream, world=1, rank=0, pg=None):
    """64 independent periodic blast patches (edges from {32,48,64,96,128} by seed), all
    advanced in one persistent launch per step under a captured graph, tile shape from the
    autotuner; each patch on its own CFL dt.  Returns zone-updates/s of the mixed path,
    beside the same batch stepped with one launch per phase per patch."""
    import torch
    from paper_1502_02935_gb300 import inputs, mhd, sharding
    allst = inputs.blast_batch(64, seed=SEED)[:args.batch]
    mine = sharding.partition([s.geom.ncell for s in allst], world)[rank]
    sts = [allst[i] for i in mine]  # this rank's share; no data crosses ranks
    cells = sum(s.geom.ncell for s in allst)
    out = {"workload": f"{args.batch} periodic blast patches, edges from {{32,48,64,96,128}} (seed 1502), gamma=5/3, "
                       "rho=1, p=0.1 / 10 inside r<0.1, |B|=1/sqrt2 along a seeded direction; mixed path",
           "cells": cells, "unit": "zone-updates/s"}
    # one context: the autotuner picks the tiles of the persistent step and then the faster
    # of the two schemes; both are timed here on the same state and tiles, the autotuned one
    # gives the value
    g = mhd.Grid(sts, precision="mixed", cfl=CFL, flags=mhd.FLAG_PERSISTENT | mhd.FLAG_GRAPH,
                 stream=stream.cuda_stream)
    cache = os.path.join(ROOT, "paper_1502_02935_gb300", "tune_cache.json")
    out["tile"] = list(g.autotune(cache, force=True))
    chosen = g.step_scheme()
    for name in ("persistent", "per_phase"):
        g.set_step_scheme(name)
        for _ in range(args.warmup):
            g.step(-1.0)
        torch.cuda.synchronize()
        l0 = g.launch_count()
        k = max(3, min(args.steps, 20))
        barrier(pg)
        ms = max_over_ranks(pg, timed_steps(g, k, stream))
        out[name] = {"value": cells * k / (ms / 1e3), "ms_per_step": ms / k, "gpu_launches": g.launch_count() - l0}
    g.close()
    out["scheme"] = chosen
    out["value"] = out[chosen]["value"]
    return out


def run_disc(args, stream):
    """Isolated gas disc (512x512x128 on 40x40x10 kpc, outflow, logarithmic potential in S,
    toroidal field with beta 10, density and temperature floors) with the thermal source:
    the plain FP64 integrator for the first 50 steps (harvesting training pairs), the
    surrogate trained on the GPU, then 150 steps of the surrogate with per-cell fallback.
    Reports the thermal phase's GPU time per step both ways (CUDA events around its kernels),
    the fallback fraction, and the L1-relative difference in T after the 150 steps against
    the plain integrator run from the same state."""
    import torch
    from paper_1502_02935_gb300 import inputs, mhd
    th = inputs.DISC_THERMAL
    nx, ny, nz = args.disc
    st = inputs.disc(nx, ny, nz)
    harvest_steps, k = args.disc_steps
    out = {"workload": f"disc {nx}x{ny}x{nz} on 40x40x10 kpc, outflow, log potential v0=220 km/s, beta=10, "
                       "T=1e4 K, floors rho>=1e-4 rho0 and 10 K<=T<=1e8 K, thermal source (stand-in cooling "
                       f"table), mixed path, {harvest_steps} plain + {k} surrogate steps",
           "cells": st.geom.ncell}
    g = mhd.Grid(st, precision="mixed", cfl=CFL, flags=mhd.FLAG_GRAPH, stream=stream.cuda_stream)
    g.set_sources(**inputs.DISC_POTENTIAL, **inputs.DISC_FLOORS)
    g.set_thermal(mhd.THERMAL_PLAIN, **th)
    # each sampled cell yields four pairs (its own and three shifted): size the stride to fill
    # the ring once
    g.surrogate_harvest(1 << 21, stride=max(1, 4 * st.geom.ncell * harvest_steps // (1 << 21)))
    g.set_profiling(True)
    for _ in range(harvest_steps):
        g.step(-1.0)
    prof = g.profile()
    g.set_profiling(False)
    plain_ms = prof["thermal"][0] / max(prof["thermal"][1], 1)
    step_ms_plain = sum(v[0] for v in prof.values()) / harvest_steps
    t0 = time.perf_counter()
    loss, rows = g.surrogate_train(epochs=100, batch=8192, lr=3e-3, seed=SEED)
    train_s = time.perf_counter() - t0
    mid = g.get_state(0)
    g.set_thermal(mhd.THERMAL_SURROGATE, **th)
    h = mhd.Grid(mid, precision="mixed", cfl=CFL, flags=mhd.FLAG_GRAPH, stream=stream.cuda_stream)
    h.set_sources(**inputs.DISC_POTENTIAL, **inputs.DISC_FLOORS)
    h.set_thermal(mhd.THERMAL_PLAIN, **th)
    del mid
    s0 = g.thermal_stats()
    g.set_profiling(True)
    for _ in range(k):
        g.step(-1.0)
        h.step(-1.0)
    prof = g.profile()
    g.set_profiling(False)
    s1 = g.thermal_stats()
    sur_ms = prof["thermal"][0] / max(prof["thermal"][1], 1)
    step_ms_sur = sum(v[0] for v in prof.values()) / k

    def temperature(x):
        bx, by, bz = x.bcc()
        kin = 0.5 * (x.U[1] ** 2 + x.U[2] ** 2 + x.U[3] ** 2) / x.U[0]
        p = (x.geom.gamma - 1) * (x.U[4] - kin - 0.5 * (bx * bx + by * by + bz * bz))
        return th["t_per_pr"] * p / x.U[0]

    Ts = temperature(g.get_state(0))
    Tp = temperature(h.get_state(0))
    floored = g.metrics()["floored"]
    g.close()
    h.close()
    out.update({"thermal_ms_plain": plain_ms, "thermal_ms_surrogate": sur_ms, "thermal_gain": plain_ms / sur_ms,
                "step_ms_plain": step_ms_plain, "step_ms_surrogate": step_ms_sur,
                "zone_updates_per_s_plain": st.geom.ncell / (step_ms_plain / 1e3),
                "zone_updates_per_s_surrogate": st.geom.ncell / (step_ms_sur / 1e3),
                "fallback_fraction": (s1["fallback"] - s0["fallback"]) / max(1, s1["cells"] - s0["cells"]),
                "floored_cells_total": floored,
                "train_rows": rows, "train_loss": loss, "train_s": train_s,
                "l1_T_vs_plain_after_%d_steps" % k: float(np.mean(np.abs(Ts - Tp)) / np.mean(np.abs(Tp)))})
    return out


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
    clocks = ClockSampler(local)
    clocks.start()
    clocks.wait_first()
    grid.step(-1.0)  # one more untimed step once the sampler runs
    torch.cuda.synchronize()
    barrier(pg)
    torch.cuda.synchronize()
    l0 = grid.launch_count()
    t_start = time.time()
    ms = timed_steps(grid, args.steps, stream)
    clk = clocks.stop(t_start, time.time())
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
    fp32_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
    fp64_peak = SM_COUNT * FP64_OPS_PER_SM_CLK * sm_max_mhz * 1e6 / 1e9
    roofs = {}
    for k, kc in KCLASS.items():
        if not prof.get(k) or not prof[k][1]:
            continue
        t = prof[k][0] / prof[k][1] / 1e3  # s per launch
        units = units_per_launch(k, n)
        cand = {
            "hbm": {"bound": "hbm", "achieved": kc["bytes"] * units / t / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "peak_note": f"{peak_kind} hbm_gbs"},
            "fp32": {"bound": "alu", "pipe": "fp32", "achieved": kc["fp32"] * units / t / 1e12, "peak": fp32_peak,
                     "unit": "TFLOP/s", "peak_note": f"FP32: 152 SMs x 128 lanes x 2 x {sm_max_mhz:.0f} MHz (derived)"},
            "fp64": {"bound": "alu", "pipe": "fp64", "achieved": kc["fp64"] * units / t / 1e9,
                     "peak": fp64_peak, "unit": "Gop/s",
                     "peak_note": f"FP64 pipe: 152 SMs x 2 ops/clk x {sm_max_mhz:.0f} MHz (derived)"},
        }
        for c in cand.values():
            c["frac"] = c["achieved"] / c["peak"]
        best = max(cand, key=lambda r: cand[r]["frac"])
        roofs[k] = dict(cand[best], others={r: round(cand[r]["frac"], 4) for r in cand if r != best})
    dom = max(roofs, key=lambda k: prof[k][0])
    # The headline roofline of the dominant kernel on the algorithmic bytes of the step's
    # definition: 128 B per cell (read the 8 FP64 fields of U^n, write those of U^n+1) times
    # the n^3 cells one launch advances, over that kernel's mean event-timed launch.
    t_dom = prof[dom][0] / prof[dom][1] / 1e3
    alg_bytes = ALG_BYTES_PER_CELL * zones
    per_point = MEASURED_DRAM_BYTES_PER_POINT.get(dom)
    roof = {"bound": "hbm", "achieved": alg_bytes / t_dom / 1e9, "peak": hbm_peak, "unit": "GB/s",
            "frac": alg_bytes / t_dom / 1e9 / hbm_peak, "kernel": dom, "launch_ms": t_dom * 1e3,
            "alg_bytes_per_launch": alg_bytes, "peak_note": f"{peak_kind} hbm_gbs",
            "traffic": per_point * units_per_launch(dom, n) if per_point else None,
            "traffic_note": MEASURED_DRAM_NOTE.get(dom),
            "step_frac": value / world * ALG_BYTES_PER_CELL / (hbm_peak * 1e9),
            "access_model": roofs[dom]}
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
    batched = run_batched(args, stream, world, rank, pg) if args.batched else None
    disc = run_disc(args, stream) if args.disc else None

    if rank != 0:
        return 0
    cb = oracle_sample(target_s=15.0) if world == 1 or rank == 0 else None
    line = {
        "metric": "zone-updates/s", "value": value, "unit": "zone-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded solenoidal turbulence, no dataset)",
        "config": dict(workload_config(n, world),
                       path="mixed precision (FP32 bulk, FP64 recovery+accumulation), graph replay",
                       l2="inputs larger than L2 (state 1.1 GB/replica, no flush)"),
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": "zone-updates/s", "h2d_bytes_per_step": io_bytes,
                "d2h_bytes_per_step": io_bytes},
        "gpu_launches": launches,
        "roofline": roof,
        "hbm_alg_frac": value / world * ALG_BYTES_PER_CELL / (hbm_peak * 1e9),
        "fp64_path": {"value": fp64_value, "unit": "zone-updates/s", "steps": k64},
        "kernel_shares": shares,
        "kernel_rooflines": roofs,
        "batched": batched,
        "disc_thermal": disc,
        "cpu_baseline": cb,
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ --table ----
def run_table(args):
    """Every workload configuration, GPU and oracle side by side (opt-in, minutes): GPU
    zone-updates/s of the plain FP64 path and the mixed path; the oracle on one host core and
    on all of them, each on a bounded sample stated in the output; and, for the 1D shock
    tube and the 2D vortex, the per-field L1 difference from the oracle at the end time."""
    import torch
    import oracle
    from paper_1502_02935_gb300 import inputs, mhd
    hbm_peak, _, _ = load_peaks()
    ncores = os.cpu_count() or 1
    stream = torch.cuda.Stream()

    def gpu_rate(states, precision, steps, flags=mhd.FLAG_GRAPH, src=None, thermal=None, riemann=None,
                 recon=None, inflow=None, scheme=None):
        sts = states if isinstance(states, list) else [states]
        g = mhd.Grid(sts if len(sts) > 1 else sts[0], precision=precision, cfl=CFL, flags=flags,
                     stream=stream.cuda_stream)
        for side, w in (inflow or {}).items():
            g.set_inflow(0, side, w)
        if riemann:
            g.set_riemann(riemann)
        if recon:
            g.set_reconstruction(recon)
        if src:
            g.set_sources(**src)
        if thermal:
            g.set_thermal(mhd.THERMAL_PLAIN, **thermal)
        if flags & mhd.FLAG_PERSISTENT:
            g.autotune(None)
            if scheme:
                g.set_step_scheme(scheme)
        for _ in range(3):
            g.step(-1.0)
        torch.cuda.synchronize()
        ms = timed_steps(g, steps, stream)
        g.close()
        return sum(st.geom.ncell for st in sts) * steps / (ms / 1e3)

    def oracle_rate(states, threads, steps, src=None, thermal=None, cfl=CFL, inflow=None):
        oracle.set_threads(threads)
        sts = states if isinstance(states, list) else [states]
        t0 = time.perf_counter()
        for st in sts:
            for _ in range(steps):
                dt = oracle.cfl_dt(st, cfl, source=src, inflow=inflow)
                st = oracle.step(st, dt, source=src, inflow=inflow)
                if thermal:
                    st, _ = oracle.thermal_apply(st, dt, thermal)
        el = time.perf_counter() - t0
        return sum(st.geom.ncell for st in sts) * steps / el, el

    def gpu_to_time(st, precision, cfl, t_end, recon=None, src=None, inflow=None):
        g = mhd.Grid(st, precision=precision, cfl=cfl, stream=stream.cuda_stream)
        if recon:
            g.set_reconstruction(recon)
        if src:
            g.set_sources(**src)
        for side, w in (inflow or {}).items():
            g.set_inflow(0, side, w)
        t, n = 0.0, 0
        while t < t_end * (1 - 1e-14):
            dt = min(g.cfl_dt(), t_end - t)
            g.step(dt)
            t += dt
            n += 1
        out = g.get_state(0)
        g.close()
        return out, n

    def l1(a, b):
        names = ["rho", "mx", "my", "mz", "E"]
        res = {nm: float(np.sum(np.abs(a.U[q] - b.U[q])) / max(np.sum(np.abs(b.U[q])), 1e-300))
               for q, nm in enumerate(names)}
        for nm in ("Bx", "By", "Bz"):
            x, y = getattr(a, nm), getattr(b, nm)
            res[nm] = float(np.sum(np.abs(x - y)) / max(np.sum(np.abs(y)), 1e-300))
        return {k: v for k, v in res.items() if np.isfinite(v)}

    table = {}
    rows = [r for r in (args.rows or "").split(",") if r]

    def want(key):
        return not rows or key in rows

    if want("C1"):
        # C1: 1D shock tube, plain FP64 only
        st = inputs.brio_wu(800)
        oracle.set_threads(ncores)
        ref, nref = oracle.run(st, 0.8, 0.1)
        t0 = time.perf_counter()
        got, n = gpu_to_time(st, "fp64", 0.8, 0.1)
        el = time.perf_counter() - t0
        r1, _ = oracle_rate(st, 1, 50, cfl=0.8)
        rn, _ = oracle_rate(st, ncores, 50, cfl=0.8)
        table["C1 Brio-Wu 800, FP64, t=0.1"] = {
            "gpu_fp64": 800 * n / el, "gpu_note": f"{n} steps with a host CFL query each (latency-bound)",
            "oracle_1core": r1, "oracle_all": rn, "steps": n, "oracle_steps": nref, "l1_fp64_vs_oracle": l1(got, ref)}
    if want("C2"):
        # C2: 2D vortex 512^2, FP64 and mixed, to t = 0.5
        st = inputs.orszag_tang(512, 512)
        oracle.set_threads(ncores)
        t0 = time.perf_counter()
        ref, nref = oracle.run(st, CFL, 0.5)
        el_ref = time.perf_counter() - t0
        g64, _ = gpu_to_time(st, "fp64", CFL, 0.5)
        gmx, _ = gpu_to_time(st, "mixed", CFL, 0.5)
        r1, _ = oracle_rate(st, 1, 10)
        table["C2 Orszag-Tang 512^2, t=0.5"] = {
            "gpu_fp64": gpu_rate(st, "fp64", 200), "gpu_mixed": gpu_rate(st, "mixed", 200),
            "oracle_1core": r1, "oracle_all": 512 * 512 * nref / el_ref, "oracle_steps": nref,
            "l1_fp64_vs_oracle": l1(g64, ref), "l1_mixed_vs_oracle": l1(gmx, ref)}
    if want("C3"):
        # C3: turbulence 256^3
        st = inputs.turbulence(256, seed=SEED)
        mixed = gpu_rate(st, "mixed", 20)
        r1, _ = oracle_rate(inputs.turbulence(64, seed=SEED), 1, 5)
        rn, _ = oracle_rate(st, ncores, 2)
        table["C3 turbulence 256^3"] = {
            "gpu_fp64": gpu_rate(st, "fp64", 5), "gpu_mixed": mixed, "hbm_alg_frac_mixed": mixed * 128 / (hbm_peak * 1e9),
            "oracle_1core": r1, "oracle_1core_sample": "64^3 box, 5 steps", "oracle_all": rn,
            "oracle_all_sample": "256^3 box, 2 steps"}
    if want("C4"):
        # C4: 64 blast patches
        sts = inputs.blast_batch(64, seed=SEED)
        r1, _ = oracle_rate(sts[:4], 1, 1)
        rn, _ = oracle_rate(sts, ncores, 1)
        table["C4 64 blast patches"] = {
            "gpu_fp64_per_phase": gpu_rate(sts, "fp64", 3),
            "gpu_mixed_per_phase": gpu_rate(sts, "mixed", 10),
            "gpu_mixed_persistent": gpu_rate(sts, "mixed", 10, flags=mhd.FLAG_GRAPH | mhd.FLAG_PERSISTENT,
                                             scheme="persistent"),
            "gpu_mixed_autotuned": gpu_rate(sts, "mixed", 10, flags=mhd.FLAG_GRAPH | mhd.FLAG_PERSISTENT),
            "oracle_1core": r1, "oracle_1core_sample": "first 4 patches, 1 step", "oracle_all": rn,
            "oracle_all_sample": "all 64 patches, 1 step"}
    if want("C5"):
        # C5: disc with the plain thermal integrator (surrogate figures: the default bench run)
        th = inputs.DISC_THERMAL
        src = dict(inputs.DISC_POTENTIAL, **inputs.DISC_FLOORS)
        st = inputs.disc(512, 512, 128)
        r1, _ = oracle_rate(inputs.disc(128, 128, 32), 1, 2, src=src, thermal=th)
        rn, _ = oracle_rate(st, ncores, 1, src=src, thermal=th)
        table["C5 disc 512x512x128, plain thermal"] = {
            "gpu_fp64": gpu_rate(st, "fp64", 3, src=src, thermal=th),
            "gpu_mixed": gpu_rate(st, "mixed", 10, src=src, thermal=th),
            "oracle_1core": r1, "oracle_1core_sample": "128x128x32 disc, 2 steps", "oracle_all": rn,
            "oracle_all_sample": "512x512x128 disc, 1 step"}
    if want("gas"):
        # pure gas dynamics (B = 0) with the solvers of Section 2.1: the 2D Sedov blast at the
        # paper's 512 x 768, and the 256^3 turbulent box without its field
        st, fl = inputs.sedov(512, 768), inputs.SEDOV_FLOORS
        oracle.set_threads(1)
        ref, ndone, el = st, 0, 0.0
        got_g = mhd.Grid(st, precision="mixed", cfl=CFL, stream=stream.cuda_stream)
        got_g.set_riemann("hllc")
        got_g.set_sources(**fl)
        for _ in range(20):
            dt = oracle.cfl_dt(ref, CFL, source=fl)
            got_g.step(dt)
            t0 = time.perf_counter()
            ref = oracle.step(ref, dt, source=fl, riemann="hllc")
            el += time.perf_counter() - t0
            ndone += 1
        got = got_g.get_state(0)
        got_g.close()
        sedov = {"gpu_mixed_" + s_: gpu_rate(st, "mixed", 50, src=fl, riemann=s_) for s_ in ("hllc", "hll", "hlld")}
        sedov["gpu_fp64_hllc"] = gpu_rate(st, "fp64", 20, src=fl, riemann="hllc")
        sedov.update({"oracle_1core_hllc": st.geom.ncell * ndone / el,
                      "oracle_1core_sample": f"512x768, {ndone} steps (one plane: the oracle's loop over z has no parallel work)",
                      "l1_mixed_hllc_vs_oracle": l1(got, ref), "l1_steps": ndone,
                      "floors": "rho >= 1e-8, p/rho >= 1e-6 (without them the plain scheme reaches p < 0 at step 7)"})
        table["Sedov 2D 512x768, B = 0 (HLLC / HLL / HLLD)"] = sedov
        st = inputs.turbulence(256, seed=SEED, b0=0.0)
        table["turbulence 256^3, B = 0 (HLLC / HLL / HLLD)"] = {
            "gpu_mixed_" + s_: gpu_rate(st, "mixed", 10, riemann=s_) for s_ in ("hllc", "hll", "hlld")}
    if want("rotor"):
        # magnetic rotor (Section 3.6) with the reconstructions of Eq. 12-14: rates at 512^2,
        # and the per-field L1 difference from the oracle at t = 0.15 on 256^2
        st = inputs.rotor(512)
        rot = {"gpu_mixed_" + r_: gpu_rate(st, "mixed", 100, recon=r_)
               for r_ in ("kappa_third", "kappa_zero", "kappa_upwind")}
        rot["gpu_fp64_kappa_third"] = gpu_rate(st, "fp64", 30)
        r1, _ = oracle_rate(st, 1, 5)
        small = inputs.rotor(256)
        oracle.set_threads(1)
        ref, nref = oracle.run(small, CFL, 0.15)
        gmx, n = gpu_to_time(small, "mixed", CFL, 0.15)
        g64, _ = gpu_to_time(small, "fp64", CFL, 0.15)
        rot.update({"oracle_1core": r1, "oracle_1core_sample": "512^2, 5 steps (one plane: no parallel work)",
                    "l1_at_t015_256sq": {"fp64": l1(g64, ref), "mixed": l1(gmx, ref)}, "steps": n,
                    "oracle_steps": nref})
        table["Rotor 2D 512^2 (kappa = 1/3, 0, -1)"] = rot
    if want("scalars"):
        # passive scalars (several gas components carried by the flow) on the 256^3 box:
        # the cost of 0, 1, 4 and 8 scalars on the mixed path
        st = inputs.turbulence(256, seed=SEED)
        row = {}
        for ns in (0, 1, 4, 8):
            g = mhd.Grid(st, precision="mixed", cfl=CFL, flags=mhd.FLAG_GRAPH, stream=stream.cuda_stream)
            if ns:
                g.set_scalars(ns)
                g.set_scalar_state(0, np.broadcast_to(st.U[0] * 0.5, (ns,) + st.U[0].shape))
            for _ in range(3):
                g.step(-1.0)
            torch.cuda.synchronize()
            ms = timed_steps(g, 10, stream)
            g.close()
            row[f"gpu_mixed_{ns}_scalars"] = st.geom.ncell * 10 / (ms / 1e3)
        small = inputs.turbulence(64, seed=SEED)
        oracle.set_threads(ncores)
        S = np.broadcast_to(small.U[0] * 0.5, (4,) + small.U[0].shape)
        t0 = time.perf_counter()
        ref = small
        for _ in range(3):
            ref, S = oracle.step_scalars(ref, S, oracle.cfl_dt(ref, CFL))
        row["oracle_all_4_scalars"] = small.geom.ncell * 3 / (time.perf_counter() - t0)
        row["oracle_sample"] = "64^3, 3 steps, 4 scalars"
        table["turbulence 256^3 with passive scalars"] = row
    if want("bow"):
        # bow shock (Section 3.3): inflow at the left, Gaussian well, 1D; to the paper's last
        # time t = 0.375
        st, src, inflow = inputs.bow_shock(400)
        oracle.set_threads(1)
        t0 = time.perf_counter()
        ref, nref = oracle.run(st, CFL, 0.375, source=src, inflow=inflow)
        el = time.perf_counter() - t0
        g64, n = gpu_to_time(st, "fp64", CFL, 0.375, src=src, inflow=inflow)
        gmx, _ = gpu_to_time(st, "mixed", CFL, 0.375, src=src, inflow=inflow)
        u = ref.U[1, 0, 0] / ref.U[0, 0, 0]
        table["Bow shock 1D 400 cells, t = 0.375"] = {
            "gpu_fp64": gpu_rate(st, "fp64", 500, src=src, inflow=inflow),
            "gpu_mixed": gpu_rate(st, "mixed", 500, src=src, inflow=inflow),
            "gpu_note": "400 cells: launch-latency-bound (graph replay)",
            "oracle_1core": 400 * nref / el, "steps": n, "oracle_steps": nref,
            "shock_x_oracle": float(st.geom.centres()[0][int(np.argmax(-np.diff(u)))]),
            "l1_vs_oracle": {"fp64": l1(g64, ref), "mixed": l1(gmx, ref)}}
    print(json.dumps({"table": table, "host_cores": ncores, "unit": "zone-updates/s"}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_CELLS, help="cells per axis (default 256)")
    ap.add_argument("--batch", type=int, default=64, help="patches of the batched workload (the first of the "
                    "64-patch seeded batch; default 64)")
    ap.add_argument("--no-batched", dest="batched", action="store_false",
                    help="skip the 64-patch batched workload")
    ap.add_argument("--disc", type=int, nargs=3, default=[512, 512, 128],
                    help="disc workload cells (nx ny nz); 0 0 0 skips it")
    ap.add_argument("--disc-steps", dest="disc_steps", type=int, nargs=2, default=[50, 150],
                    help="disc workload: plain (harvest) steps, then surrogate steps")
    ap.add_argument("--table", action="store_true",
                    help="every workload configuration, GPU and oracle side by side (minutes; no bench line)")
    ap.add_argument("--rows", default="",
                    help="with --table: comma-separated subset of C1,C2,C3,C4,C5,gas,rotor,bow,scalars (default all)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.table:
        return run_table(args)
    if args.disc == [0, 0, 0]:
        args.disc = None
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
