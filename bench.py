"""Benchmark of the coupled LB-MPCD step on the 2D channel workload.

Workload: D2Q9 2048 x 512 channel (tau 0.8, g 1e-7, FP32 deviation storage),
MPCD on the central 256 LB columns at refinement 2 (512 x 1020 cells, 10
particles per cell, 5,222,400 particles), SRD 130 degrees, kT 1e-4, 2-column
coupling buffers with the windowed MPCD -> LB feedback (W = 100).  One step =
LB stream-collide (whose launch also builds the previous step's collision-cell
table and applies its MPCD -> LB imposition) + particle pass.  Synthetic data
only.

Prints one JSON line.  The device-timed value comes from CUDA events around
lbmpcd_step(K) (graph replay) on the handle's stream, bracketed by a barrier
and a synchronize; the per-kernel roofline from a second, per-kernel-event
profiled run; e2e through the C ABI with host buffers.  --impl reference times
the FP64 CPU oracle on the same workload (bounded sample) instead.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(
    name="channel2d_2048x512_fp32",
    params=dict(lattice=9, nx=2048, ny=512, nz=1, tau=0.8, force=(1e-7, 0.0, 0.0), refine=2,
                ppc=10, alpha=math.radians(130.0), kT=1e-4, mass=1.0, coupling_width=2,
                precision=1, feedback=1, window=100, resample_density=0, seed=2),
    region=(896, 1152))

# 3D slab channel, FP32: D3Q19 256x128x128, tau 0.9, g 5e-8; MPCD slab x in
# [112,144) at refinement 2 (64 x 252 x 256 cells, 41,287,680 particles),
# SRD about random axes at 120 degrees, kT 1e-4.
SLAB = dict(
    name="slab3d_256x128x128_fp32",
    params=dict(lattice=19, nx=256, ny=128, nz=128, tau=0.9, force=(5e-8, 0.0, 0.0), refine=2,
                ppc=10, alpha=math.radians(120.0), kT=1e-4, mass=1.0, coupling_width=2,
                precision=1, feedback=1, window=100, resample_density=0, seed=3),
    region=(112, 144))


def ensemble_workload():
    """The 64-replica uneven ensemble of tests/inputs.py (Ny in {16,32,64,128},
    Nx = 4 Ny, r in {1,2,4}, tau ~ U[0.6,1.2], g ~ U[1e-7,1e-6], 5..20 particles
    per cell, MPCD on the central Nx/4 columns): 29,056,224 particles and
    1,626,112 LB nodes in one handle."""
    from tests import inputs
    return inputs.ensemble_replicas()


def rank_params(params: dict, rank: int) -> dict:
    """The channel of rank r under torchrun: the same workload with seed + 1000 r,
    so that the ranks run independent replicas (no collective on the data path)."""
    return dict(params, seed=params["seed"] + 1000 * rank)


def max_over_ranks(value: float, world: int, device) -> float:
    """The slowest rank's value (a MAX all-reduce; every rank calls it)."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(steps: int, world: int, seconds: float) -> float:
    """Whole-job steps/s: the steps of all ranks over the slowest rank's time."""
    return world * steps / seconds


METRIC = "coupled_steps_per_s"
UNIT = "steps/s"
PROFILE_NOTE = os.path.join(ROOT, "profiles", "ncu_particle_pass_channel2048x512.md")


def algorithmic_bytes(p, region):
    """Algorithmic HBM bytes per step of each kernel (FP32 storage, 2D): per LB
    node 2 q 4 B (9 populations read and written), per particle its state read
    and written (home 4 + offsets 8 + velocities 8, and the id 4 that keys the
    MPCD-AT random velocity), per collision cell 2 (4 + 4 d) B = 24 B (count and
    momentum sums written by the binning and read back for the table).  The
    cell-table items run in the LB launch, so their bytes count there."""
    nx, ny, r, ppc = p["nx"], p["ny"], p["refine"], p["ppc"]
    fluid = nx * (ny - 2)
    Wx, Hy = (region[1] - region[0]) * r, (ny - 2) * r
    npart = Wx * Hy * ppc
    ncell = Wx * (Hy + 1)
    return dict(
        lb_pull=72 * fluid + 24 * ncell,
        particle_pass=(44 if p.get("collision", 0) else 40) * npart,
        lb_rows=72 * fluid, cell_items=24 * ncell,   # the two halves of lb_pull in the overlapped form
        fluid_nodes=fluid, particles=npart, cells=ncell)


def step_launches(n0: int, last_sort: int, steps: int, mode: int, kchunk: int = 64, overlapped: bool = False):
    """Kernel launches of lbmpcd_step(steps) from step n0 (the library's chunk
    rule: chunks of 64 steps, then one of the rest; a counting sort of
    four kernels before a chunk once 64 steps have passed since the last one;
    one prep kernel per chunk; two kernels per step, or in the overlapped form
    one LB launch per chunk and three kernels per step but the last (particle
    pass, next LB update beside it, table + a8), or one persistent kernel per
    chunk).  Returns (launches, step count, last sort)."""
    n, left, total = n0, steps, 0
    while left > 0:
        kc = min(kchunk, left)
        if n - last_sort >= kchunk:
            total += 4
            last_sort = n
        total += 1 + (1 if mode == 1 else (3 * kc if overlapped else 2 * kc))
        n += kc
        left -= kc
    return total, n, last_sort


def n_chunks(steps: int, kchunk: int = 64) -> int:
    """Chunks of lbmpcd_step(steps): 64 steps each, then the rest."""
    return -(-steps // kchunk)


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
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
        self.f.flush()
        rows = [ln.split(",") for ln in open(self.f.name).read().strip().splitlines() if ln.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def ncu_traffic_per_launch(pair: bool = False):
    """DRAM bytes per launch from the committed ncu summary, if the kernel
    sources are unchanged since the capture (hashes recorded in the summary):
    the particle pass, or with pair=True the particle pass plus the LB rows
    launched beside it (each captured alone: ncu serialises launches)."""
    import hashlib
    try:
        txt = open(PROFILE_NOTE).read()
    except Exception:
        return None
    vals = {}
    for ln in txt.splitlines():
        if ": " in ln and ln.strip().startswith("- "):
            k, v = ln.strip()[2:].split(": ", 1)
            vals[k.strip()] = v.strip()
    for f in ("mpcd.cu", "lb.cu", "lb_core.cuh", "cell_core.cuh", "common.cuh", "kernels.h"):
        src = open(os.path.join(ROOT, "paper_2004_00304_gb300", "csrc", f), "rb").read()
        if vals.get(f + " sha256[:16]") != hashlib.sha256(src).hexdigest()[:16]:
            return None
    try:
        t = float(vals["dram_bytes_per_launch"])
        return t + float(vals["rows_dram_bytes_per_launch"]) if pair else t
    except Exception:
        return None


def _time_oracle(omp: bool, seconds: float):
    import oracle
    s = oracle.OracleSim(WORKLOAD["params"], omp=omp)
    s.set_region(*WORKLOAD["region"])
    s.step(1)                       # warm-up
    t0 = time.perf_counter()
    n = 0
    while True:
        s.step(1)
        n += 1
        if time.perf_counter() - t0 > seconds:
            break
    return n, time.perf_counter() - t0


def cpu_baseline(seconds: float = 12.0):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload
    (full coupled steps of the whole 2048 x 512 system): on all host cores
    (its OpenMP build: LB nodes, particle streaming and redraw shared out, the
    rest serial) and single-threaded."""
    import oracle
    n1, dt1 = _time_oracle(False, seconds)
    nm, dtm = _time_oracle(True, seconds)
    threads = oracle.num_threads(True)
    return {"value": nm / dtm, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{nm} full coupled steps of the {WORKLOAD['name']} workload (5.2M particles) after 1 "
                      f"warm-up step, FP64, {threads} threads (OpenMP over LB nodes, streaming and redraw), "
                      f"{dtm:.1f} s",
            "single_thread": {"value": n1 / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"{n1} full coupled steps, FP64, one thread, {dt1:.1f} s"}}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    # the oracle on all host cores (its OpenMP build; the results do not depend
    # on the thread count)
    s = oracle.OracleSim(WORKLOAD["params"], omp=True)
    threads = oracle.num_threads(True)
    s.set_region(*WORKLOAD["region"])
    t = time.perf_counter()
    s.step(1)
    t_step = time.perf_counter() - t
    budget = 90.0
    nwarm = min(args.warmup, max(0, int(10.0 / t_step)))
    s.step(nwarm)
    ntimed = max(1, min(args.steps, int(budget / max(t_step, 1e-6))))
    t0 = time.perf_counter()
    s.step(ntimed)
    dt = time.perf_counter() - t0
    v = ntimed / dt
    sample = (f"{ntimed} timed full coupled steps (of {args.steps} requested) after {nwarm + 1} warm-up "
              f"steps, FP64 oracle, {threads} threads (OpenMP over LB nodes, streaming and redraw)")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": ntimed, "warmup": nwarm + 1, "ms_per_step": 1e3 * dt / ntimed,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD["name"]},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist
    import __graft_entry__
    import paper_2004_00304_gb300 as lb

    __graft_entry__.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    params = rank_params(WORKLOAD["params"], rank)
    p = WORKLOAD["params"]
    ab = algorithmic_bytes(p, WORKLOAD["region"])

    def barrier():
        if world > 1:
            dist.barrier()

    with torch.cuda.stream(stream):
        sim = lb.Lbmpcd(params, stream=stream)
        sim.set_region(0, *WORKLOAD["region"])
        launch = choose_launch(sim, args)
        # keep a copy of the initial state on the host (pinned) for the e2e leg
        names = ("POPS", "PART_POS", "PART_VEL", "PART_HOME")
        host_in = {}
        for nm in names:
            n = lb.lbmpcd_field_size(sim._h, 0, nm)
            t = torch.empty(n, dtype=torch.int32 if nm in lb.INT_FIELDS else torch.float64, pin_memory=True)
            sim.get(nm, out=t.numpy())
            host_in[nm] = t
        # the overlapped form (the default per-kernel form where it applies)
        ov = launch["mode"] == 0 and not launch.get("serial") and not launch.get("lb_tma")
        # the clock sampler starts before the warm-up steps, so that the timed
        # steps follow the warm-up without an idle gap (an idle GPU takes some
        # microseconds to come back to full speed)
        sampler = ClockSampler(local_rank) if rank == 0 else None
        time.sleep(0.3 if sampler else 0)
        sim.step(args.warmup)
        stream.synchronize()
        _, n_w, sort_w = step_launches(0, 0, args.warmup, launch["mode"], overlapped=ov)

        # ---- device-timed region: K steps of graph replay -----------------
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clocks = sampler.stop() if sampler else None
        ms = e0.elapsed_time(e1)
        launches, _, _ = step_launches(n_w, sort_w, args.steps, launch["mode"], overlapped=ov)
        ms = max_over_ranks(ms, world, dev)

        # ---- per-kernel durations (events around every launch) ------------
        kprof = min(args.steps, 640)
        phase_ms, nlaunch = sim.step_profiled(kprof)
        if ov:   # per step: the pass with the next LB update beside it, then the table + a8 launch
            nchunk = n_chunks(kprof)
            per_launch = {"particle_pass+lb_rows": phase_ms["particle_pass"] / kprof,
                          "cell_items": phase_ms["cell_pass"] / kprof,
                          "lb_pull (first of a chunk)": phase_ms["lb_pull"] / max(nchunk, 1)}
        else:
            per_launch = {k: phase_ms[k] / kprof for k in ("lb_pull", "particle_pass")}

        # ---- e2e through the C ABI with host buffers ----------------------
        e2e = None
        if not args.no_e2e:
            out_u = torch.empty(lb.lbmpcd_field_size(sim._h, 0, "U"), dtype=torch.float64, pin_memory=True)
            out_v = torch.empty(lb.lbmpcd_field_size(sim._h, 0, "PART_VEL"), dtype=torch.float64,
                                pin_memory=True)
            sim2 = lb.Lbmpcd(params, stream=stream)
            sim2.set_region(0, *WORKLOAD["region"])
            # warm-up of the same calls: the handle's staging buffer is
            # allocated by the first host-side set / get
            for nm in names:
                sim2.set(nm, host_in[nm])
            sim2.step(args.warmup)
            sim2.get("U", out=out_u.numpy())
            sim2.get("PART_VEL", out=out_v.numpy())
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            for nm in names:
                sim2.set(nm, host_in[nm])
            sim2.step(args.steps)
            sim2.get("U", out=out_u.numpy())
            sim2.get("PART_VEL", out=out_v.numpy())
            torch.cuda.synchronize()
            t_e2e = time.perf_counter() - t0
            barrier()
            t_e2e = max_over_ranks(t_e2e, world, dev)
            h2d = sum(t.numel() * t.element_size() for t in host_in.values())
            d2h = out_u.numel() * 8 + out_v.numel() * 8
            e2e = {"value": job_rate(args.steps, world, t_e2e), "unit": UNIT,
                   "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                   "note": "set_state of the full initial state from pinned host memory, K steps, "
                           "get_fields of U and particle velocities to pinned host memory"}
            sim2.close()
        sim.close()

    if rank != 0:
        return
    steps_per_s = job_rate(args.steps, world, ms * 1e-3)
    peaks = measured_peaks()
    hbm = float(peaks["hbm_gbs"]) if peaks else 6800.0
    step_bytes = ab["lb_pull"] + ab["particle_pass"]
    if ov:
        # the dominant unit is the particle pass with the LB update of the next
        # step running beside it: their bytes over the time of the pair
        dom = "particle_pass+lb_rows"
        kb = {dom: ab["particle_pass"] + ab["lb_rows"], "cell_items": ab["cell_items"],
              "lb_pull (first of a chunk)": ab["lb_rows"]}
        traffic = ncu_traffic_per_launch(pair=True) if not p.get("collision", 0) else None
    else:
        dom = "particle_pass"
        kb = {"lb_pull": ab["lb_pull"], "particle_pass": ab["particle_pass"]}
        traffic = ncu_traffic_per_launch() if not p.get("collision", 0) else None
    t_dom = per_launch[dom] * 1e-3
    achieved = kb[dom] / t_dom / 1e9
    kernels = {}
    for k in kb:
        t = per_launch[k] * 1e-3
        kernels[k] = {"us_per_launch": per_launch[k] * 1e3, "algorithmic_bytes": kb[k],
                      "achieved_gbs": kb[k] / t / 1e9 if t > 0 else None,
                      "frac_of_measured_hbm": (kb[k] / t / 1e9) / hbm if t > 0 else None}
    out = {
        "metric": METRIC, "value": steps_per_s, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD["name"], "lb_nodes": f"{p['nx']}x{p['ny']}",
                   "particles": ab["particles"], "collision_cells": ab["cells"],
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "working set ~300 MB per step > 129 MB L2 (no flush needed)", "launch": launch},
        "lb_mlups": ab["fluid_nodes"] * steps_per_s / 1e6,
        "mpcd_mparticle_upd_per_s": ab["particles"] * steps_per_s / 1e6,
        "step_hbm": {"algorithmic_bytes_per_step": step_bytes,
                     "achieved_gbs": step_bytes * steps_per_s / world / 1e9,
                     "frac_of_measured": step_bytes * steps_per_s / world / 1e9 / hbm,
                     "frac_of_nominal_7900": step_bytes * steps_per_s / world / 1e9 / 7900.0},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic,
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback 6.8 TB/s"},
        "kernels": kernels,
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": e2e,
    }
    if not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline()
    print(json.dumps(out), flush=True)


def run_slab3d(args):
    """Secondary measurement: the 3D slab channel (D3Q19, 41.3M particles)."""
    import torch
    import __graft_entry__
    import paper_2004_00304_gb300 as lb
    __graft_entry__.build()
    p, (x0, x1) = SLAB["params"], SLAB["region"]
    r = p["refine"]
    fluid = p["nx"] * (p["ny"] - 2) * p["nz"]
    Wx, Hy, Wz = (x1 - x0) * r, (p["ny"] - 2) * r, p["nz"] * r
    parts, cells = Wx * Hy * Wz * p["ppc"], Wx * (Hy + 1) * Wz
    ab = dict(lb_pull=152 * fluid + 32 * cells,   # 19 populations read + 19 written, 4 B each; cell
                                                  # sums 2 (4 + 4 d) B, built in the same launch
              particle_pass=56 * parts)           # home 4 + offsets 12 + velocities 12, read and written
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim = lb.Lbmpcd(p, stream=stream)
        sim.set_region(0, x0, x1)
        launch = choose_launch(sim, args)
        sim.step(args.warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        kprof = 64
        phase_ms, _ = sim.step_profiled(kprof)
        sim.close()
    sps = args.steps / (ms * 1e-3)
    peaks = measured_peaks()
    hbm = float(peaks["hbm_gbs"]) if peaks else 6800.0
    step_bytes = ab["lb_pull"] + ab["particle_pass"]
    kernels = {}
    if launch["mode"] == 0 and not launch.get("serial") and not launch.get("lb_tma"):
        # overlapped: per step the pass with the next step's LB rows beside it, then the table + a8 launch
        kb = {"particle_pass+lb_rows": (ab["particle_pass"] + 152 * fluid, phase_ms["particle_pass"] / kprof),
              "cell_items": (32 * cells, phase_ms["cell_pass"] / kprof)}
    else:
        kb = {k: (ab[k], phase_ms[k] / kprof) for k in ("lb_pull", "particle_pass")}
    for k, (b, t_ms) in kb.items():
        t = t_ms * 1e-3
        kernels[k] = {"us_per_launch": t * 1e6, "algorithmic_bytes": b, "achieved_gbs": b / t / 1e9,
                      "frac_of_measured_hbm": b / t / 1e9 / hbm}
    out = {"metric": METRIC, "value": sps, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": SLAB["name"], "lb_nodes": f"{p['nx']}x{p['ny']}x{p['nz']}", "particles": parts,
                      "collision_cells": cells, "launch": launch},
           "lb_mlups": fluid * sps / 1e6, "mpcd_mparticle_upd_per_s": parts * sps / 1e6,
           "step_hbm": {"algorithmic_bytes_per_step": step_bytes, "achieved_gbs": step_bytes * sps / 1e9,
                        "frac_of_measured": step_bytes * sps / 1e9 / hbm},
           "kernels": kernels}
    print(json.dumps(out), flush=True)


def choose_launch(sim, args) -> dict:
    """The launch form of the step: autotuned on a copy of the handle (default),
    or forced to per-kernel graphs / the persistent kernel."""
    if args.launch == "auto":
        return sim.autotune(steps=256)
    mode = 1 if args.launch == "persistent" else 0
    tma = args.launch == "graphs_tma"
    sim.set_launch_mode(mode, lb_tma=tma)
    return dict(mode=mode, blocks_per_sm=0, lb_nodes_per_thread=None, lb_tma=tma, candidates=1)


def run_ensemble(args):
    """Secondary measurement: the 64-replica uneven ensemble in one handle
    (one launch per kernel and step covering every replica, 64-step graphs)."""
    import torch
    import __graft_entry__
    import paper_2004_00304_gb300 as lb
    __graft_entry__.build()
    reps = ensemble_workload()
    if args.fp16:
        for r in reps:
            r["params"] = dict(r["params"], precision=2)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim = lb.Lbmpcd([r["params"] for r in reps], stream=stream)
        for k, r in enumerate(reps):
            sim.set_region(k, *r["region"])
        launch = choose_launch(sim, args)
        sim.step(args.warmup)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        kprof = 64
        phase_ms, _ = sim.step_profiled(kprof)   # events around every launch group
        sim.close()
    phases_us = {k: v * 1e3 / kprof for k, v in phase_ms.items() if v}
    sps = args.steps / (ms * 1e-3)
    nodes = sum(r["params"]["nx"] * (r["params"]["ny"] - 2) for r in reps)
    parts = sum((r["region"][1] - r["region"][0]) * r["params"]["refine"] * (r["params"]["ny"] - 2) * r["params"]["refine"]
                * r["params"]["ppc"] for r in reps)
    cells = sum((r["region"][1] - r["region"][0]) * r["params"]["refine"] * ((r["params"]["ny"] - 2) * r["params"]["refine"] + 1)
                for r in reps)
    pop_b = 36 if args.fp16 else 72
    step_bytes = pop_b * nodes + 40 * parts + 24 * cells
    peaks = measured_peaks()
    hbm = float(peaks["hbm_gbs"]) if peaks else 6800.0
    out = {"metric": METRIC, "value": sps, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f16-storage/f32" if args.fp16 else "f32", "data": "synthetic",
           "config": {"workload": "ensemble64_uneven_" + ("fp16dev" if args.fp16 else "fp32"), "replicas": len(reps),
                      "lb_nodes": nodes, "particles": parts, "launch": launch},
           "lb_mlups": nodes * sps / 1e6, "mpcd_mparticle_upd_per_s": parts * sps / 1e6,
           "step_hbm": {"algorithmic_bytes_per_step": step_bytes, "achieved_gbs": step_bytes * sps / 1e9,
                        "frac_of_measured": step_bytes * sps / 1e9 / hbm},
           "phases_us_per_step_profiled": phases_us}
    print(json.dumps(out), flush=True)


def _ensemble_running_means(lb, CT, cfg, mode, theta, replicas, burn, steps, every, seed0=0):
    """Running means over time and `replicas` channels (distinct seeds, one
    handle) of (a) the velocity imposed on the two inner-buffer columns (the
    MPCD -> LB feedback, from the populations there) and (b) the x-averaged
    LB velocity profile, after each sample; samples `every` steps apart from
    `burn` steps on.  Returns numpy arrays [samples][ny - 2][2] and
    [samples][ny - 2]."""
    import numpy as np
    import torch
    name, fb, window, K = mode
    p0, (x0, x1) = cfg["params"], cfg["region"]
    nx, ny = p0["nx"], p0["ny"]
    ps = [dict(p0, feedback=fb, window=window, seed=p0["seed"] + seed0 + 7919 * r) for r in range(replicas)]
    sim = lb.Lbmpcd(ps)
    for r in range(replicas):
        sim.set_region(r, x0, x1)
        CT.start_from_poiseuille(sim, r, dict(cfg, params=ps[r]))
    if fb == 2:
        sim.set_closure(theta, interval=K)
    sim.step(burn)
    cols = [x0 + 1, x1 - 2]                      # inner-buffer columns (coupling width 2)
    cxs = torch.tensor([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=torch.float64, device="cuda")
    uf = torch.empty(3 * ny * nx, dtype=torch.float64, device="cuda")
    pops = torch.empty(9 * ny * nx, dtype=torch.float64, device="cuda")
    S = steps // every
    acc_lb = torch.zeros(ny - 2, dtype=torch.float64, device="cuda")
    acc_imp = torch.zeros(ny - 2, 2, dtype=torch.float64, device="cuda")
    m_lb = torch.empty(S, ny - 2, dtype=torch.float64, device="cuda")
    m_imp = torch.empty(S, ny - 2, 2, dtype=torch.float64, device="cuda")
    for k in range(S):
        sim.step(every)
        for r in range(replicas):
            sim.get("U", r, out=uf)
            acc_lb += uf.view(3, ny, nx)[0, 1:ny - 1, :].mean(dim=1)
            sim.get("POPS", r, out=pops)
            f = pops.view(9, ny, nx)[:, 1:ny - 1, cols]
            acc_imp += (cxs[:, None, None] * f).sum(0) / f.sum(0)
        m_lb[k] = acc_lb / ((k + 1) * replicas)
        m_imp[k] = acc_imp / ((k + 1) * replicas)
    sim.close()
    return m_imp.cpu().numpy(), m_lb.cpu().numpy()


def _rel_err(a, b):
    """Relative L2 distance per sample: a, b [samples][...]."""
    import numpy as np
    ax = tuple(range(1, a.ndim))
    return np.sqrt(((a - b) ** 2).sum(axis=ax) / (b ** 2).sum(axis=ax))


def _startup_profile(yw, t, H, g, nu, terms=200):
    """Plane Poiseuille flow started from rest under a constant force g: the
    steady parabola minus its decaying odd sine modes (yw from the wall,
    channel height H, kinematic viscosity nu)."""
    import numpy as np
    u = g * yw * (H - yw) / (2 * nu)
    for n in range(1, 2 * terms, 2):
        u = u - 4 * g * H * H / (nu * np.pi ** 3 * n ** 3) * np.sin(n * np.pi * yw / H) * \
            np.exp(-(n * np.pi / H) ** 2 * nu * t)
    return u


def _transient_imposed_error(lb, CT, cfg, mode, theta, replicas, steps, every):
    """`replicas` channels (distinct seeds, one handle) start from rest under
    the force; every `every` steps the velocity imposed on the two
    inner-buffer columns, averaged over the replicas (no time average: the
    flow is changing), is compared with the start-up solution at that time.
    Returns (relative L2 errors per sample, device seconds of the steps)."""
    import numpy as np
    import torch
    name, fb, window, K = mode
    p0, (x0, x1) = cfg["params"], cfg["region"]
    nx, ny = p0["nx"], p0["ny"]
    ps = [dict(p0, feedback=fb, window=window, seed=p0["seed"] + 7919 * r) for r in range(replicas)]
    sim = lb.Lbmpcd(ps)
    for r in range(replicas):
        sim.set_region(r, x0, x1)
    if fb == 2:
        sim.set_closure(theta, interval=K)
    nu = (p0["tau"] - 0.5) / 3.0
    yw = np.arange(1, ny - 1) + 0.5 - 1.0
    cols = [x0 + 1, x1 - 2]
    cxs = torch.tensor([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=torch.float64, device="cuda")
    pops = torch.empty(9 * ny * nx, dtype=torch.float64, device="cuda")
    errs, t_dev = [], 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in range(steps // every):
        e0.record()
        sim.step(every)
        e1.record()
        torch.cuda.synchronize()
        t_dev += e0.elapsed_time(e1) * 1e-3
        acc = torch.zeros(ny - 2, 2, dtype=torch.float64, device="cuda")
        for r in range(replicas):
            sim.get("POPS", r, out=pops)
            f = pops.view(9, ny, nx)[:, 1:ny - 1, cols]
            acc += (cxs[:, None, None] * f).sum(0) / f.sum(0)
        u = (acc / replicas).cpu().numpy()
        ua = _startup_profile(yw, (k + 1) * every, ny - 2, p0["force"][0], nu)
        errs.append(float(np.linalg.norm(u - ua[:, None]) / np.linalg.norm(np.repeat(ua[:, None], 2, 1))))
    sim.close()
    return np.asarray(errs), t_dev


def _time_to(errs, every, tol=0.01):
    """Steps after which the running-mean error stays at or below tol (None if
    it is above tol at the last sample)."""
    import numpy as np
    above = np.nonzero(errs > tol)[0]
    k_ok = 0 if above.size == 0 else int(above[-1]) + 1
    return None if k_ok >= errs.size else (k_ok + 1) * every


def run_closure(args):
    """Secondary measurement: the learned closure on the 1024 x 256 channel
    (MPCD on the central 128 LB columns at refinement 2, g = 1e-7), with the
    LB viscosity matched to the SRD fluid's (tau = matched_tau) so that the
    coupled steady state is the analytic Poiseuille profile.  The network is
    trained here on data the coupled method generates (16 channels of the
    same family at Ny in {64,...,512}, g in [1e-7, 1e-6]); its gain over the
    plain 8-frame mean is measured on held-out channels.  The channel then
    runs with the plain windowed coupling (W = 100 and W = 8) and with the
    closure (inference every step and every 8 steps).

    Speed: steps/s of one channel, CUDA events around `steps` steps.
    Accuracy and time to solution: every mode runs 8 replicas (distinct
    seeds) from the Poiseuille profile for 1000 steps; then, every 10 steps
    for 5000 steps, the running mean over time and replicas of the velocity
    imposed on the inner-buffer columns (the averaged MPCD -> LB feedback)
    and of the x-averaged LB profile is taken.  A mode's error is measured
    against the plain W = 100 coupling: an independent 16-replica W = 100 run over
    the same window, whose running means at the same times are the
    reference (the MPCD mean at the buffer differs from the analytic profile
    by ~1 % and drifts slowly, the same in every mode).  A mode's time to
    solution is the number of channel-steps (steps x replicas) after which
    its imposed-profile error against that reference stays at or below 1 %,
    over its measured single-channel step rate (null if it is above 1 % at
    the end); the errors against the analytic profile are given beside.

    Transient (surrogate_speedup_to_1pct): 64 replicas of a 256 x 64 channel
    start from rest under g = 3.2e-6; every 50 steps the replica-mean
    velocity imposed on the inner-buffer columns is compared with the
    start-up solution of plane Poiseuille flow at that time (the viscosities
    matched, the coupled channel is one fluid).  A window of W steps lags the
    accelerating flow by ~W/2 steps; the closure's 8 frames by ~4.  Time to
    solution = steps until the error stays at or below 1 %, times the
    handle's measured step time; the speedup is W = 100's over the
    closure's at K = 8.
    """
    import numpy as np
    import torch
    import __graft_entry__
    import paper_2004_00304_gb300 as lb
    from paper_2004_00304_gb300 import closure_train as CT
    __graft_entry__.build()
    t0 = time.time()
    tau = CT.matched_tau(10, 1e-4, 130 * math.pi / 180.0, 2)
    X, T = CT.generate(CT.training_channels(16, seed=1, tau=tau), spinup=1500, samples=150, every=10)
    Xv, Tv = CT.generate(CT.training_channels(4, seed=2, tau=tau), spinup=1500, samples=20, every=25)
    t1 = time.time()
    train_steps, batch = 8000, 128
    theta, losses = CT.train(X, T, steps=train_steps, batch=batch, lr=1e-3, seed=0)
    torch.cuda.synchronize()
    t2 = time.time()
    ev = CT.evaluate(theta, Xv, Tv)
    n_train = int(X.shape[0])
    del X, T, Xv, Tv

    cfg = CT.channel(256, 1e-7, seed=5, nx=1024, region_cols=128, tau=tau)
    p0, (x0, x1) = cfg["params"], cfg["region"]
    nx, ny = p0["nx"], p0["ny"]
    modes = [("plain_W100", 1, 100, 0), ("plain_W8", 1, 8, 0), ("closure_K1", 2, 100, 1), ("closure_K8", 2, 100, 8)]
    runs = {}
    peaks = measured_peaks()
    R, burn, n_acc, every = 8, 1000, 5000, 10
    ref_imp, ref_lb = _ensemble_running_means(lb, CT, cfg, modes[0], None, 16, burn, n_acc, every, seed0=100_000)
    u_ref = CT.poiseuille(np.arange(1, ny - 1) + 0.5, ny, p0["tau"], p0["force"][0])
    for name, fb, window, K in modes:
        pm = dict(p0, feedback=fb, window=window)
        sim = lb.Lbmpcd([pm])
        sim.set_region(0, x0, x1)
        CT.start_from_poiseuille(sim, 0, dict(cfg, params=pm))
        if fb == 2:
            sim.set_closure(theta, interval=K)
        sim.step(max(args.warmup, 1000))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sim.step(args.steps)
        e1.record()
        torch.cuda.synchronize()
        run = {"steps_per_s": args.steps / (e0.elapsed_time(e1) * 1e-3)}
        if fb == 2 and K == 1:
            ph, _ = sim.step_profiled(64)
            t_launch = ph["closure"] / 64 * 1e-3                 # one closure_step launch per step
            P = 2 * (-(-((ny - 2) * p0["refine"]) // 16))
            flops = P * 45.7e6
            peak = float(peaks["bf16_tflops_sustained"]) if peaks else 1700.0   # timed inside the step
            run["closure_step"] = {"patches": P, "us_per_launch": t_launch * 1e6,
                                   "roofline": {"bound": "tensor", "achieved": flops / t_launch / 1e12, "peak": peak,
                                                "unit": "TFLOP/s", "frac": flops / t_launch / 1e12 / peak}}
        sim.close()
        im, ml = _ensemble_running_means(lb, CT, cfg, (name, fb, window, K), theta, R, burn, n_acc, every)
        e_imp, e_lb = _rel_err(im, ref_imp), _rel_err(ml, ref_lb)
        steps_to = _time_to(e_imp, every)
        pick = lambda e: {str((k + 1) * every): float(e[k]) for k in (0, 9, 49, 99, 249, 499) if k < e.size}
        run["ensemble"] = {"replicas": R, "burn_in": burn, "sample_every": every,
                           "imposed_err_vs_W100_ref": pick(e_imp), "lb_err_vs_W100_ref": pick(e_lb),
                           "imposed_err_vs_poiseuille": pick(_rel_err(im, np.broadcast_to(u_ref[None, :, None], im.shape))),
                           "lb_err_vs_poiseuille": pick(_rel_err(ml, np.broadcast_to(u_ref[None, :], ml.shape))),
                           "steps_to_1pct_imposed": steps_to, "steps_to_1pct_lb": _time_to(e_lb, every),
                           "seconds_to_1pct": None if steps_to is None else steps_to * R / run["steps_per_s"]}
        runs[name] = run
    # start-up transient: 64 replicas of a 256 x 64 channel from rest, where a
    # window's lag (W / 2 steps) costs accuracy while the flow accelerates
    tcfg = CT.channel(64, 3.2e-6, seed=9, nx=256, region_cols=32, tau=tau)
    transient = {"workload": "64 replicas, 256x64 D2Q9, MPCD central 32 columns at r = 2, g = 3.2e-6, from rest",
                 "replicas": 64, "steps": 6000, "sample_every": 50}
    tmodes = [("plain_W8", 1, 8, 0), ("plain_W25", 1, 25, 0), ("plain_W100", 1, 100, 0),
              ("closure_K1", 2, 100, 1), ("closure_K8", 2, 100, 8)]
    for name, fb, window, K in tmodes:
        errs, t_dev = _transient_imposed_error(lb, CT, tcfg, (name, fb, window, K), theta, 64, 6000, 50)
        steps_to = _time_to(errs, 50)
        transient[name] = {"imposed_err_at_steps": {str((k + 1) * 50): float(errs[k]) for k in (1, 9, 19, 39, 59, 79, 99, 119)},
                           "mean_err_last_half": float(errs[errs.size // 2:].mean()),
                           "steps_to_1pct": steps_to, "step_s": t_dev / 6000,
                           "seconds_to_1pct": None if steps_to is None else steps_to * t_dev / 6000}
    tw, tc = transient["plain_W100"]["seconds_to_1pct"], transient["closure_K8"]["seconds_to_1pct"]
    t_w, t_c = runs["plain_W100"]["ensemble"]["seconds_to_1pct"], runs["closure_K8"]["ensemble"]["seconds_to_1pct"]
    out = {"metric": METRIC, "value": runs["closure_K8"]["steps_per_s"], "unit": UNIT, "n_gpus": 1,
           "steps": args.steps, "warmup": max(args.warmup, 1000),
           "ms_per_step": 1e3 / runs["closure_K8"]["steps_per_s"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32 (network bf16/f32-acc)", "data": "synthetic",
           "config": {"workload": "channel2d_1024x256_closure_fp32", "lb_nodes": f"{nx}x{ny}",
                      "mpcd_region_cols": x1 - x0, "refine": p0["refine"], "ppc": p0["ppc"], "tau": tau,
                      "g": p0["force"][0]},
           "closure": {"training": {"patches": n_train, "steps": train_steps, "batch": batch,
                                    "data_s": t1 - t0, "train_s": t2 - t1,
                                    "patches_per_s": train_steps * batch / (t2 - t1),
                                    "loss_first20": float(losses[:20].mean()), "loss_last100": float(losses[-100:].mean())},
                       "heldout": {k: [float(v) for v in ev[k]] for k in ("rmse_net", "rmse_mean8", "gain")},
                       "in_loop": runs,
                       "step_time_over_plain_W100": runs["plain_W100"]["steps_per_s"] / runs["closure_K8"]["steps_per_s"],
                       "transient": transient,
                       "transient_err_W100_over_K8": transient["plain_W100"]["mean_err_last_half"] /
                                                     transient["closure_K8"]["mean_err_last_half"],
                       "surrogate_speedup_to_1pct": (tw / tc) if (tw and tc) else None,
                       "surrogate_speedup_to_1pct_steady": (t_w / t_c) if (t_w and t_c) else None}}
    print(json.dumps(out), flush=True)


def run_closure_kernel(args):
    """The 1024 x 256 channel with the closure evaluated every step (network
    parameters of the initial distribution: the kernels' cost does not depend
    on their values); for kernel profiling."""
    import torch
    import __graft_entry__
    import paper_2004_00304_gb300 as lb
    from paper_2004_00304_gb300 import closure_train as CT
    __graft_entry__.build()
    cfg = CT.channel(256, 1e-7, seed=5, nx=1024, region_cols=128)
    sim = lb.Lbmpcd([cfg["params"]])
    sim.set_region(0, *cfg["region"])
    sim.set_closure(CT.init_params(0), interval=1)
    sim.step(args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    sim.step(args.steps)
    e1.record()
    torch.cuda.synchronize()
    sps = args.steps / (e0.elapsed_time(e1) * 1e-3)
    # closure_step alone: event-timed per launch (64 patches, 45.7 MFLOP each)
    kprof = min(args.steps, 256)
    ph, _ = sim.step_profiled(kprof)
    t_cl = ph["closure"] / kprof * 1e-3
    npatch = 2 * (-(-((cfg["params"]["ny"] - 2) * cfg["params"]["refine"]) // 16))
    flops = 45.7e6 * npatch
    peaks = measured_peaks()
    sus = float(peaks["bf16_tflops_sustained"]) if peaks else 1700.0
    print(json.dumps({"metric": METRIC, "value": sps, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
                      "warmup": args.warmup, "higher_is_better": True, "data": "synthetic",
                      "config": {"workload": "channel2d_1024x256_closure_every_step_fp32"},
                      "closure_step": {"us_per_launch": t_cl * 1e6, "patches": npatch,
                                       "tflops": flops / t_cl / 1e12,
                                       "frac_of_sustained_bf16": flops / t_cl / 1e12 / sus,
                                       "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained" if peaks
                                       else "fallback 1.7 PFLOP/s"}}), flush=True)
    sim.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="channel",
                    choices=["channel", "ensemble", "closure", "closure_kernel", "slab3d"],
                    help="channel: the 2048x512 headline workload; ensemble: the 64-replica ensemble; "
                         "closure: training, gain and in-loop runs of the learned closure (extra lines)")
    ap.add_argument("--fp16", action="store_true", help="ensemble only: FP16 deviation storage")
    ap.add_argument("--collision", default="srd", choices=["srd", "at"],
                    help="channel only: SRD (Eq. 4, default) or MPCD-AT (Eq. 6) collisions (extra line)")
    ap.add_argument("--launch", default="auto", choices=["auto", "graphs", "graphs_tma", "persistent"],
                    help="launch form of the step: autotuned (default), per-kernel graphs, persistent kernel")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.collision == "at":
        global WORKLOAD
        WORKLOAD = dict(WORKLOAD, name=WORKLOAD["name"] + "_mpcd_at", params=dict(WORKLOAD["params"], collision=1))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "ensemble":
        run_ensemble(args)
        return
    if args.workload == "closure":
        run_closure(args)
        return
    if args.workload == "closure_kernel":
        run_closure_kernel(args)
        return
    if args.workload == "slab3d":
        run_slab3d(args)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
