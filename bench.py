#!/usr/bin/env python
"""Throughput of the mechanical-interaction step (agent-steps/s).

Workload (the paper's benchmark B at GB300 size): 4,194,304 cells with centres
uniform in a cube sized for a mean of 8 overlapping neighbours, diameters
U[8, 12], maximum displacement 0 (benchmark B's rule), 20 fused steps with the
grid rebuilt every step.  One bench step = those 20 steps, so it processes
4,194,304 * 20 agent-steps.  Before each timed step a 256 MB buffer is written
to flush the 129 MB L2 (outside the step's CUDA events).

Prints one JSON line (rank 0).  --impl reference times the FP64 oracle on the
host cores instead (a bounded sample of the same workload per bench step).

Multi-GPU: the path is weak-scaled as independent replicas (each rank runs its
own population; no collective on the data path); the barrier and the max over
ranks only frame the timing.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

N_AGENTS = 1 << 22
MEAN_NEIGHBOURS = 8.0
POP_SEED = 8                        # rank r uses POP_SEED + 1000 r
SIM_STEPS = 20
WORKLOAD = ("density cube: 4,194,304 cells, centres uniform in a cube sized for a mean of 8 "
            "overlapping neighbours, d U[8,12], max displacement 0; 20 fused steps (grid rebuilt "
            "every step) per bench step")
BYTES_PER_AGENT_SWEEP = 32          # sweep + move: read 16 B row, write 16 B row
BYTES_PER_AGENT_STEP = 88           # whole step (grid bin 16, scatter 40, sweep 32)
BYTES_PER_BOX = 12
# algorithmic FP32 operations of the method: distance pre-test per candidate in
# the 27 surrounding boxes (3 sub, 3 mul/fma, 1 add, 1 mul, 1 compare), Eq. 1 per
# contact (delta: sqrt + sub; R: mul, add, div; sqrt(R delta): mul + sqrt; phi:
# 2 mul + sub; direction: div + 3 mul; sum: 3 add) and the displacement per
# agent (|F|, mass, dt/m, 3 mul, |v|, cap test, 3 add)
FLOPS_PER_CANDIDATE = 9
FLOPS_PER_CONTACT = 17
FLOPS_PER_AGENT = 25
# FP32 roof (derived: MEASURED_PEAKS.json has no FP32 figure): 152 SMs x 128
# FP32 lanes x 2 flop (FMA) x 2.07 GHz; issue roof: 4 schedulers per SM, one
# warp instruction each per clock
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
ISSUE_PEAK_GINST_S = 152 * 4 * 2.07
# One launch of the sweep on this workload under ncu (cache flushed): DRAM bytes
# read + written and warp instructions executed.  They describe the sweep's
# source as it was captured (sha256[:16] of the files below) and are reported
# as null once that source changes.
SWEEP_SOURCES = ("ug_sweep2.cu", "ug_internal.cuh")
SWEEP_CAPTURE = {"src": "88518fcd5b8d6723", "dram_bytes": 95_005_440 + 38_936_832, "warp_inst": 575_849_854}


def sweep_source_hash() -> str:
    h = hashlib.sha256()
    for f in SWEEP_SOURCES:
        with open(os.path.join(ROOT, "paper_2105_00039_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def sweep_capture():
    """The captured counters if the sweep's source is unchanged since, else None."""
    if SWEEP_CAPTURE["src"] is None or SWEEP_CAPTURE["src"] != sweep_source_hash():
        return None
    return SWEEP_CAPTURE


def issue_roofline(avg_launch_ms: float):
    """The sweep against the instruction-issue limit, or None without a current
    capture of its instruction count."""
    cap = sweep_capture()
    if cap is None:
        return None
    achieved = cap["warp_inst"] / (avg_launch_ms / 1000.0) / 1e9
    return {"warp_inst_per_launch": cap["warp_inst"], "achieved_ginst_s": achieved,
            "peak_ginst_s": ISSUE_PEAK_GINST_S, "frac": achieved / ISSUE_PEAK_GINST_S,
            "peak_source": "derived: 152 SMs x 4 schedulers x 1 warp instruction per clock "
                           "x 2.07 GHz; instructions per launch from ncu"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the density, batched, adjoint and comparison rows")
    return ap.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def reduce_max(pg, value: float, device=None) -> float:
    """Max of a per-rank float over all ranks (identity without a process group)."""
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock/throttle samples taken while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------- CPU oracle
def _oracle_chunk(args):
    """One process's share of a sampled oracle step: the population is rebuilt
    from its seed, the oracle's sampled step (its own kd-tree over all cells,
    then the listed cells against every cell) is timed.  With the GPU's forces
    of the same cells (rows F_x, F_y, F_z, contacts, by cell index) it also
    returns, after the timing, each cell's condition-scaled force error
    |F_gpu - F| / max(|F|, S) (S: the sum of the pair terms' magnitudes) and
    the number of cells whose contact count differs."""
    n, nbar, seed, lo, hi, stride, gpu = args
    import oracle as O
    from paper_2105_00039_gb300 import populations as P
    st = P.density_cube(n, nbar, seed=seed)
    idx = np.arange(lo, hi, stride, dtype=np.int64)
    t0 = time.perf_counter()
    ref = O.step_sampled(st, idx, O.Params(max_disp=0.0))
    secs = time.perf_counter() - t0
    if gpu is None:
        return len(idx), secs, None
    F, S = ref["F"], ref["S"]
    scale = np.maximum(np.linalg.norm(F, axis=1), S)
    diff = np.linalg.norm(gpu[:, :3].astype(np.float64) - F, axis=1)
    err = np.where(scale > 0, diff / np.where(scale > 0, scale, 1.0), 0.0).astype(np.float32)
    count_bad = int(np.sum(gpu[:, 3].astype(np.int64) != ref["npairs"]))
    return len(idx), secs, (err, count_bad)


class OraclePool:
    """The FP64 oracle on the host's cores: `procs` spawned processes (spawn, so
    that no CUDA state is inherited), each running the oracle as it stands on
    its own slice of the cells."""

    def __init__(self, procs: int):
        import multiprocessing as mp
        self.procs = procs
        self.pool = mp.get_context("spawn").Pool(procs) if procs > 1 else None

    def step(self, n, nbar, seed, fraction=1.0, gpu=None):
        """One sampled step over `fraction` of the cells (every cell when 1):
        returns (cells evaluated, wall seconds of the slowest process, and with
        `gpu` (n x 4 float32, by cell index) the per-cell force errors and the
        count of contact-count mismatches, else None)."""
        stride = max(1, int(round(1.0 / fraction)))
        per = (n + self.procs - 1) // self.procs
        jobs = [(n, nbar, seed, p * per, min(n, (p + 1) * per), stride,
                 None if gpu is None else gpu[p * per:min(n, (p + 1) * per):stride])
                for p in range(self.procs)]
        res = self.pool.map(_oracle_chunk, jobs) if self.pool else [_oracle_chunk(jobs[0])]
        cmp = None
        if gpu is not None:
            cmp = (np.concatenate([r[2][0] for r in res]), sum(r[2][1] for r in res))
        return sum(r[0] for r in res), max(r[1] for r in res), cmp

    def close(self):
        if self.pool:
            self.pool.close()
            self.pool.join()


def cpu_oracle_baseline(gpu_forces=None):
    """The oracle on all host cores (one full step of every cell, split over
    the cores) and on one core (a sample of the cells, its kd-tree included).
    With the GPU's forces of the same population it also returns the parity
    of every cell's force and contact count against that oracle step (else
    None in their place)."""
    cores = os.cpu_count() or 1
    pool = OraclePool(cores)
    try:
        cells, secs, cmp = pool.step(N_AGENTS, MEAN_NEIGHBOURS, POP_SEED, gpu=gpu_forces)
    finally:
        pool.close()
    parity = None
    if cmp is not None:
        err, count_bad = cmp
        parity = {"workload": "the headline population's first step, every cell",
                  "force_condition_scaled": {"max": float(err.max()),
                                             "median": float(np.median(err)),
                                             "cells": int(err.size), "tolerance": 1e-5},
                  "contact_counts_differing": count_bad,
                  "oracle": "FP64, kd-tree pair search (the same run as cpu_baseline)"}
    one = OraclePool(1)
    cells1, secs1, _ = one.step(N_AGENTS, MEAN_NEIGHBOURS, POP_SEED, fraction=1.0 / 8.0)
    pinning = "none (the OS scheduler places the processes)"
    return parity, {"value": cells / secs, "unit": "agent-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"one FP64 oracle step of all {cells} cells of the bench workload, split over "
                      f"{cores} spawned processes (each builds its own kd-tree over all cells); "
                      f"slowest process {secs:.1f} s",
            "pinning": pinning,
            "one_core": {"value": cells1 / secs1, "unit": "agent-steps/s", "cores": 1,
                         "sample": f"every 8th cell ({cells1} cells) against all cells, kd-tree "
                                   f"included, {secs1:.1f} s"}}


def run_reference(args, world, rank, pg):
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    pool = OraclePool(cores)
    frac = 0.5
    try:
        for _ in range(args.warmup):
            pool.step(N_AGENTS, MEAN_NEIGHBOURS, POP_SEED, frac)
        cells, total = 0, 0.0
        for _ in range(args.steps):
            c, dt, _ = pool.step(N_AGENTS, MEAN_NEIGHBOURS, POP_SEED, frac)
            cells += c
            total += dt
    finally:
        pool.close()
    value = cells / total if total > 0 else 0.0
    line = {
        "impl": "reference", "metric": "agent-steps/s", "value": value, "unit": "agent-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * total / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_agents": N_AGENTS,
                   "sample": "every 2nd cell against all cells per bench step (one oracle step)",
                   "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "agent-steps/s", "cores": cores, "kind": "oracle",
                         "sample": f"every 2nd cell of the 4,194,304 against all cells per bench step, "
                                   f"split over {cores} spawned processes, kd-tree built in each"},
        "e2e": {"value": value, "unit": "agent-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- measurement
def candidates_and_contacts(U, x, prm):
    """Mean candidates (agents in the 27 surrounding boxes, self excluded),
    contacts per agent and the number of boxes of a population, from the
    library's grid and forces.  Measurement only: the box counts are summed
    over 3x3x3 neighbourhoods with torch on the per-box table."""
    import torch
    srt, perm, start, info, _ = U.grid_build(x, contact_margin=prm.contact_margin)
    g = U.grid_info_from_bytes(info)
    dx, dy, dz = g["dims"]
    cnt = (start[1:g["nboxes"] + 1] - start[:g["nboxes"]]).to(torch.float64).reshape(dz, dy, dx)
    nb = torch.nn.functional.conv3d(cnt[None, None], torch.ones(1, 1, 3, 3, 3, dtype=torch.float64,
                                                                   device=cnt.device), padding=1)[0, 0]
    n = x.shape[0]
    cand = float((cnt * nb).sum().item() - n) / n
    F = U.compute_forces(srt, start, info, prm)
    return cand, float(F[:, 3].double().mean().item()), int(g["nboxes"])


def forces_by_row(U, x, prm):
    """The library's forces of every row of x (F_x, F_y, F_z, contacts), by row,
    on the host."""
    srt, perm, start, info, _ = U.grid_build(x, contact_margin=prm.contact_margin)
    F = U.compute_forces(srt, start, info, prm)
    out = np.empty((x.shape[0], 4), np.float32)
    out[perm.cpu().numpy().astype(np.int64)] = F.cpu().numpy()
    return out


def _timed(fn, reps, flush=None):
    """Mean milliseconds of fn() over reps runs, CUDA events on the current
    stream, L2 flushed before each run (outside the events)."""
    import torch
    stream = torch.cuda.current_stream()
    tot = 0.0
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        tot += a.elapsed_time(b)
    return tot / reps


class Population:
    """One population on the device with a Stepper sized for it, and the
    three ways of stepping it the rows below compare."""

    def __init__(self, U, st, prm, dev, slack=1.05):
        import torch
        self.U, self.prm = U, prm
        self.n = len(st)
        self.x0 = torch.from_numpy(st).to(dev)
        self.mb = U.estimate_max_boxes(self.x0, prm.contact_margin, slack=slack)
        self.sp = U.Stepper(self.n, self.mb, dev)
        self.x = torch.empty_like(self.x0)
        self.perm = torch.empty(self.n, dtype=torch.int32, device=dev)
        self.lib = U.load()
        self.one = torch.tensor([0, self.n], dtype=torch.int32, device=dev)
        self.pdev = prm.as_tensor(dev)[None]
        self.walks = {}
        for name, walk in (("full_runs", 1), ("windows_always", 2)):
            t = U.ug_tuning()
            t.agents_per_lane, t.sweep_block, t.neighbour_walk = 2, 128, walk
            self.walks[name] = t

    def reset(self):
        self.x.copy_(self.x0)
        self.U._check(self.lib.ug_iota(self.U._ptr(self.perm), self.n, self.U._stream()), "ug_iota")

    def run(self, nsteps, how="default"):
        """ug_step ("default": neighbour-row windows where they pay), every pair
        once, or one simulation through ug_step_batched walking the full runs
        or the windows at every grid density."""
        self.reset()
        if how == "default":
            self.sp.step(self.x, self.perm, self.prm, nsteps)
        elif how == "pairs_once":
            self.sp.step(self.x, self.perm, self.prm, nsteps, pairs_once=True)
        else:
            self.sp.step_batched(self.x, self.perm, self.one, self.pdev, nsteps, self.walks[how])

    def traced(self, nsteps, events):
        self.reset()
        self.sp.step_traced(self.x, self.perm, self.prm, nsteps, events)


def kernel_split(pop, nsteps, reps=1):
    """Per-kernel device time per step (us), from ug_step_traced (events
    between the kernels, which also un-chains them)."""
    import torch
    names = ("key", "scan", "place", "canon", "sweep")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 + 5 * nsteps)]
    for e in ev:
        e.record()
    split = {nm: 0.0 for nm in ("bounds",) + names}
    for _ in range(reps):
        pop.traced(nsteps, ev)
        ev[-1].synchronize()
        split["bounds"] += ev[0].elapsed_time(ev[1])
        for t in range(nsteps):
            for j, nm in enumerate(names):
                split[nm] += ev[1 + 5 * t + j].elapsed_time(ev[2 + 5 * t + j])
    pop.sp.check("traced")
    return {k: 1000.0 * v / (reps * (1 if k == "bounds" else nsteps)) for k, v in split.items()}


def density_row(U, dev, flush, hbm, n, nbar, nsteps=SIM_STEPS, reps=2, seed=None):
    """One Benchmark-B style population: agent-steps/s with ug_step, with the
    full three-box runs, with the windows at any density, and with every pair
    once; the kernel split, and the step's and the sweep's rooflines."""
    from paper_2105_00039_gb300 import populations as P
    prm = U.Params(max_disp=0.0)
    pop = Population(U, P.density_cube(n, float(nbar), seed=nbar if seed is None else seed), prm, dev)
    out = {"n_agents": n, "mean_neighbours_target": nbar}
    for how in ("default", "full_runs", "windows_always", "pairs_once"):
        pop.run(nsteps, how)
        pop.sp.check(how)
        ms = _timed(lambda: pop.run(nsteps, how), reps, flush)
        pop.sp.check(how)
        out[how] = {"agent_steps_per_s": n * nsteps / (ms / 1e3), "ms_per_step": ms / nsteps}
    split = kernel_split(pop, nsteps)
    cand, cont, boxes = candidates_and_contacts(U, pop.x0, prm)
    per_step_s = out["default"]["ms_per_step"] / 1e3
    alg = BYTES_PER_AGENT_STEP * n + BYTES_PER_BOX * boxes
    flops = n * (FLOPS_PER_CANDIDATE * cand + FLOPS_PER_CONTACT * cont + FLOPS_PER_AGENT)
    tflops = flops / (split["sweep"] * 1e-6) / 1e12
    out.update({"step_alg_gbs": alg / per_step_s / 1e9, "step_hbm_frac": alg / per_step_s / 1e9 / hbm,
                "boxes": boxes, "candidates_per_agent": cand, "contacts_per_agent": cont,
                "sweep_alu_tflops": tflops, "sweep_alu_frac": tflops / FP32_PEAK_TFLOPS,
                "windows_speedup_over_full_runs": out["full_runs"]["ms_per_step"] /
                                                  out["windows_always"]["ms_per_step"],
                "kernel_us_per_step_traced": split})
    return out


def run_ours(args, world, rank, local, pg):
    import torch

    from paper_2105_00039_gb300 import populations as P
    from paper_2105_00039_gb300 import ugmech as U

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    st = P.density_cube(N_AGENTS, MEAN_NEIGHBOURS, seed=POP_SEED + 1000 * rank)
    n = len(st)
    prm = U.Params(max_disp=0.0)
    pop = Population(U, st, prm, dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        hbm = float(json.load(f)["hbm_gbs"])

    for _ in range(args.warmup):
        pop.run(SIM_STEPS)
    pop.sp.check("warm-up")
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if pg is not None:
        pg.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        # the metric: K bench steps (kernels chained with programmatic dependent
        # launch), each preceded by an L2 flush outside its events
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            pop.run(SIM_STEPS)
            ends[k].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        # per-kernel durations: the same bench steps with events between kernels
        split = kernel_split(pop, SIM_STEPS, reps=args.steps)
        torch.cuda.synchronize()
    if pg is not None:
        pg.barrier()
    pop.sp.check("timed steps")
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    tot_ms = reduce_max(pg, sum(step_ms), dev)
    ms_per_step = tot_ms / args.steps
    value = world * n * SIM_STEPS * args.steps / (tot_ms / 1000.0)

    # roofline of the dominant kernel (the sweep), per launch, and of the step
    avg_launch_ms = split["sweep"] / 1000.0
    cand, cont, boxes = candidates_and_contacts(U, pop.x0, prm)   # frozen population
    # the GPU's forces of the population, compared with the oracle's step in the
    # CPU baseline leg
    gpu_forces = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        gpu_forces = forces_by_row(U, pop.x0, prm)
    alg_flops = n * (FLOPS_PER_CANDIDATE * cand + FLOPS_PER_CONTACT * cont + FLOPS_PER_AGENT)
    alu_tflops = alg_flops / (avg_launch_ms / 1000.0) / 1e12
    sweep_bytes = BYTES_PER_AGENT_SWEEP * n
    step_alg = BYTES_PER_AGENT_STEP * n + BYTES_PER_BOX * boxes
    step_gbs = step_alg / (ms_per_step / SIM_STEPS / 1000.0) / 1e9
    cap = sweep_capture()

    line = {
        "metric": "agent-steps/s", "value": value, "unit": "agent-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_agents": n, "mean_neighbours": MEAN_NEIGHBOURS,
                   "sim_steps_per_step": SIM_STEPS, "boxes": boxes, "max_boxes": pop.mb,
                   "l2": "flushed (256 MB write) before each timed step, outside its events",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "alu", "kernel": "sweep", "achieved": alu_tflops,
                     "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": alu_tflops / FP32_PEAK_TFLOPS,
                     "traffic": cap["dram_bytes"] if cap else None,
                     "avg_launch_us": avg_launch_ms * 1000.0,
                     "alg_flops_per_launch": alg_flops,
                     "candidates_per_agent": cand, "contacts_per_agent": cont,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz "
                                    "(MEASURED_PEAKS.json has no FP32 figure)",
                     "issue": issue_roofline(avg_launch_ms),
                     "hbm": {"achieved_gbs": sweep_bytes / (avg_launch_ms / 1000.0) / 1e9,
                             "peak_gbs": hbm, "alg_bytes_per_launch": sweep_bytes,
                             "frac": sweep_bytes / (avg_launch_ms / 1000.0) / 1e9 / hbm,
                             "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"},
                     "step_alg_bytes": step_alg, "step_alg_gbs": step_gbs,
                     "step_hbm_frac": step_gbs / hbm},
        "kernel_us_per_step_traced": split,
        "kernel_share": {k: v / sum(split.values()) for k, v in split.items()},
        "gpu_launches": args.steps * (2 + 6 * SIM_STEPS),
        "clocks": clk.summary(),
        "wall_s_timed_region": wall,
    }

    # end to end through the public API: pinned host rows in, rows (by id) out
    if not args.no_e2e:
        sim = U.Simulation(n, pop.mb, dev)
        host_in = torch.from_numpy(st).pin_memory()
        host_out = torch.empty((n, 4), dtype=torch.float32).pin_memory()
        for _ in range(2):
            sim.run(host_in, prm, SIM_STEPS, host_out)
        torch.cuda.synchronize()
        e_ms = 0.0
        for _ in range(args.steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim.run(host_in, prm, SIM_STEPS, host_out)
            b.record(stream)
            b.synchronize()
            e_ms += a.elapsed_time(b)
        sim.stepper.check("e2e")
        e_ms = reduce_max(pg, e_ms, dev)
        line["e2e"] = {"value": world * n * SIM_STEPS * args.steps / (e_ms / 1000.0),
                       "unit": "agent-steps/s", "h2d_bytes_per_step": 16 * n,
                       "d2h_bytes_per_step": 16 * n}
        del sim

    # the extra rows and the CPU baselines are single-GPU measurements: a
    # multi-GPU run reports only the headline
    if not args.no_extras and world == 1:
        walk = {"workload": "the headline population, the same steps",
                "default_ms_per_step": ms_per_step / SIM_STEPS}
        for how in ("full_runs", "windows_always"):
            pop.run(SIM_STEPS, how)
            pop.sp.check(how)
            walk[how + "_ms_per_step"] = _timed(lambda: pop.run(SIM_STEPS, how), args.steps, flush) / SIM_STEPS
        line["walk"] = walk
        del pop
        torch.cuda.empty_cache()
        line["density_sweep"] = measure_density(U, dev, flush, hbm)
        line["lattice_1m"] = measure_lattice(U, dev, flush, hbm)
        line["batched"] = measure_batched(dev, flush)
        line["adjoint"] = measure_adjoint(dev, flush)
        line["version_ladder"] = measure_ladder(dev, flush)
        line["pairs_once"] = measure_pairs_once(dev, flush)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["parity"], line["cpu_baseline"] = cpu_oracle_baseline(gpu_forces)
        line["cpu_grid_baseline"] = cpu_grid_rate(st, 10)
    if rank == 0:
        print(json.dumps(line), flush=True)


def cpu_grid_rate(st, nsteps):
    """The paper's CPU uniform-grid method (baseline/cpu_ug: float64, linked-list
    grid rebuilt every step, OpenMP over agents) on all host cores: the CPU
    comparison the paper's speedups are quoted against."""
    try:
        sys.path.insert(0, os.path.join(ROOT, "baseline", "cpu_ug"))
        import cpu_ug
        threads = cpu_ug.max_threads()
        _, secs = cpu_ug.steps(st, nsteps, threads=threads)
    except Exception as e:   # no g++ / OpenMP on this host
        return {"unavailable": f"{type(e).__name__}: {e}"[:200]}
    return {"value": len(st) * nsteps / secs, "unit": "agent-steps/s", "cores": threads,
            "kind": "cpu uniform grid, float64, OpenMP",
            "sample": f"{nsteps} steps of all {len(st)} cells ({secs:.2f} s)"}


# ---------------------------------------------------------------------------- extra rows
def measure_density(U, dev, flush, hbm):
    """Benchmark-B style density sweep: 4,194,304 cells at a mean of 2, 8, 32, 64
    overlapping neighbours and 16,777,216 at 12 (the out-of-cache run), max
    displacement 0, 20 steps each."""
    import torch
    rows = []
    for n, nbar in ((1 << 22, 2), (1 << 22, 8), (1 << 22, 32), (1 << 22, 64), (1 << 24, 12)):
        rows.append(density_row(U, dev, flush, hbm, n, nbar))
        torch.cuda.empty_cache()
    return rows


def measure_lattice(U, dev, flush, hbm, nsteps=100, reps=2):
    """2^20 cells on the jittered 102^3 lattice (spacing 9, jitter 1.5, d U[9,11]),
    100 fused steps with the default displacement rules, without and with a
    contact margin of 1.5 (the variant that reaches ~12 overlapping neighbours)."""
    from paper_2105_00039_gb300 import populations as P
    st = P.lattice_1m(0)
    n = len(st)
    out = {"workload": "2^20 cells, first sites of a 102^3 lattice (spacing 9, jitter 1.5, d U[9,11]), "
                       f"{nsteps} fused steps"}
    for name, margin in (("margin_0", 0.0), ("margin_1.5", 1.5)):
        prm = U.Params(contact_margin=margin)
        pop = Population(U, st, prm, dev, slack=1.2)
        row = {}
        for how in ("default", "windows_always"):
            pop.run(nsteps, how)
            pop.sp.check(how)
            ms = _timed(lambda: pop.run(nsteps, how), reps, flush)
            pop.sp.check(how)
            row[how] = {"agent_steps_per_s": n * nsteps / (ms / 1e3), "ms_per_step": ms / nsteps}
        cand, cont, boxes = candidates_and_contacts(U, pop.x0, prm)
        alg = BYTES_PER_AGENT_STEP * n + BYTES_PER_BOX * boxes
        row.update({"contacts_per_agent_initial": cont, "candidates_per_agent_initial": cand,
                    "step_hbm_frac": alg / (row["default"]["ms_per_step"] / 1e3) / 1e9 / hbm,
                    "kernel_us_per_step_traced": kernel_split(pop, nsteps)})
        out[name] = row
    return out


def measure_batched(dev, flush, nsims=256, nsteps=50, reps=3):
    """256 independent simulations (agent counts log-uniform in [1e3, 2e5], mean
    neighbours U[4, 40]), 50 steps: the batched step as one CUDA graph (the
    library's BatchedGraph) against the 256 simulations run one after another
    with the plain step of the same method, both as one CUDA graph and launched
    call by call."""
    import torch

    from paper_2105_00039_gb300 import populations as P
    from paper_2105_00039_gb300 import ugmech as U
    st, offs = P.batched_population(nsims=nsims, seed=0)
    n = len(st)
    x0 = torch.from_numpy(st).to(dev)
    offs_t = torch.from_numpy(offs.astype(np.int32)).to(dev)
    prm = U.Params()
    pdev = torch.stack([prm.as_tensor(dev) for _ in range(nsims)])
    parts = [x0[int(offs[k]):int(offs[k + 1])] for k in range(nsims)]
    # generous per-simulation box capacity: dense random clouds expand while relaxing
    caps = [4 * U.estimate_max_boxes(p, 0.0, slack=1.0, extra_extent=24.0) + 1000 for p in parts]
    mb = int(sum(caps))
    sp = U.Stepper(n, mb, dev, nsims=nsims)
    x = torch.empty_like(x0)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    tune = U.tune_batched(x0, offs_t, pdev, nsims, mb)
    lib = U.load()

    def reset():
        x.copy_(x0)
        U._check(lib.ug_iota(U._ptr(perm), n, U._stream()), "ug_iota")

    reset()
    graph = U.BatchedGraph(sp, x, perm, offs_t, pdev, nsteps, tune)

    def run_graph():
        reset()
        graph.replay()
    run_graph()
    sp.check("batched")
    t_batched = _timed(run_graph, reps, flush)
    sp.check("batched")
    # sequential plain runs, each simulation with its own workspace
    steppers = [U.Stepper(len(p), caps[k], dev) for k, p in enumerate(parts)]
    xs = [torch.empty_like(p) for p in parts]
    ps = [torch.empty(len(p), dtype=torch.int32, device=dev) for p in parts]

    def sequential():
        for k in range(nsims):
            xs[k].copy_(parts[k])
            U._check(lib.ug_iota(U._ptr(ps[k]), len(parts[k]), U._stream()), "ug_iota")
            steppers[k].step(xs[k], ps[k], prm, nsteps, pairs_once=bool(tune.pair_mode))
    sequential()
    torch.cuda.synchronize()
    t_seq = _timed(sequential, reps, flush)
    for k in range(0, nsims, 37):
        steppers[k].check("sequential")
    same = all(torch.equal(x[int(offs[k]):int(offs[k + 1])], xs[k]) for k in range(nsims))
    # the same sequential runs captured as one CUDA graph (launch overhead removed)
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream())
    gseq = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(gseq, stream=side):
            sequential()
    torch.cuda.current_stream().wait_stream(side)
    gseq.replay()
    torch.cuda.synchronize()
    t_seq_graph = _timed(gseq.replay, reps, flush)
    for k in range(0, nsims, 37):
        steppers[k].check("sequential graph")
    same_graph = all(torch.equal(x[int(offs[k]):int(offs[k + 1])], xs[k]) for k in range(nsims))
    return {"workload": f"{nsims} simulations, {n} agents in total, {nsteps} steps",
            "batched_graph_ms": t_batched, "sequential_plain_ms": t_seq,
            "sequential_graph_ms": t_seq_graph,
            "batched_agent_steps_per_s": n * nsteps / (t_batched / 1e3),
            "sequential_agent_steps_per_s": n * nsteps / (t_seq / 1e3),
            "sequential_graph_agent_steps_per_s": n * nsteps / (t_seq_graph / 1e3),
            "speedup_vs_sequential_calls": t_seq / t_batched,
            "speedup_vs_sequential_graph": t_seq_graph / t_batched,
            "bit_identical_to_plain": bool(same and same_graph),
            "tuned_sweep_block": int(tune.sweep_block),
            "tuned_agents_per_lane": int(tune.agents_per_lane),
            "tuned_pair_mode": int(tune.pair_mode),
            "tuned_neighbour_walk": int(tune.neighbour_walk)}


def measure_adjoint(dev, flush, side=64, nsteps=50, ckpt=10, reps=3):
    """Differentiable workload: side^3 lattice cells, 50 steps, checkpoints every
    10; forward (checkpointed) and backward (ug_step_backward per segment)."""
    import torch

    from paper_2105_00039_gb300 import populations as P
    from paper_2105_00039_gb300 import ugmech as U
    from paper_2105_00039_gb300.autograd import trajectory
    st = P.lattice_cube(side, seed=5)
    x0 = torch.from_numpy(st).to(dev)
    tgt = x0[:, :3] + 0.1
    prm = U.Params(adherence=0.0)
    mb = U.estimate_max_boxes(x0, 0.0, slack=2.0)
    state = {}

    def fwd():
        x = x0.clone().requires_grad_(True)
        k = torch.tensor(2.0, requires_grad=True)
        gm = torch.tensor(1.0, requires_grad=True)
        out = trajectory(x, k, gm, prm, nsteps, ckpt, mb)
        state["loss"] = ((out[:, :3] - tgt) ** 2).mean()
        state["leaves"] = (x, k, gm)

    def bwd():
        state["loss"].backward()

    fwd(); bwd(); torch.cuda.synchronize()
    f_ms, b_ms = 0.0, 0.0
    for _ in range(reps):
        f_ms += _timed(fwd, 1, flush)
        b_ms += _timed(bwd, 1, flush)
    f_ms /= reps
    b_ms /= reps
    # the plain forward alone (no checkpoint copies, no autograd) for reference
    sp = U.Stepper(len(st), mb, dev)
    x = torch.empty_like(x0)
    perm = torch.empty(len(st), dtype=torch.int32, device=dev)
    lib = U.load()

    def plain():
        x.copy_(x0)
        U._check(lib.ug_iota(U._ptr(perm), len(st), U._stream()), "ug_iota")
        sp.step(x, perm, prm, nsteps)
    plain(); torch.cuda.synchronize()
    p_ms = _timed(plain, reps, flush)
    return {"workload": f"{side}^3 = {side ** 3} lattice cells, {nsteps} steps, checkpoint every {ckpt}",
            "forward_ms": f_ms, "backward_ms": b_ms, "plain_forward_ms": p_ms,
            "backward_over_forward": b_ms / f_ms, "backward_over_plain_forward": b_ms / p_ms}


def measure_pairs_once(dev, flush, reps=5):
    """Newton's third law (ug_forces_symmetric) on the box-sorted 2^20-cell
    lattice: one force evaluation with every pair evaluated once (forward half
    of each neighbourhood, fixed-point atomics to both agents), the same walk
    over all 27 boxes, and the main path's force sweep (ug_compute_forces)."""
    from paper_2105_00039_gb300 import populations as P
    from paper_2105_00039_gb300 import ugmech as U
    import torch
    x = torch.from_numpy(P.lattice_1m(0)).to(dev)
    n = x.shape[0]
    prm = U.Params()
    lib = U.load()
    srt, perm, start, info, status = U.grid_build(x)
    F = torch.empty_like(srt)
    ws = U.workspace(32 * n + 256, dev)
    out = {"workload": "2^20-cell lattice, box-sorted; one force evaluation (grid built beforehand)"}

    def sym(once):
        U._check(lib.ug_forces_symmetric(once, U._ptr(srt), U._ptr(start), U._ptr(info), n, prm.c(),
                                         U._ptr(F), U._ptr(ws), ws.numel(), U._ptr(status),
                                         U._stream()), "ug_forces_symmetric")

    def main():
        U._check(lib.ug_compute_forces(U._ptr(srt), U._ptr(start), U._ptr(info), n, prm.c(), U._ptr(F),
                                       U._ptr(status), U._stream()), "ug_compute_forces")
    for name, fn in (("pairs_once_fixed_point", lambda: sym(1)),
                     ("pairs_from_both_sides_same_walk", lambda: sym(0)),
                     ("main_path_force_sweep", main)):
        fn()
        U.check_status(status, name)
        ms = _timed(fn, reps, flush)
        U.check_status(status, name)
        out[name] = {"ms": ms, "agents_per_s": n / (ms / 1e3)}
    return out


def measure_ladder(dev, flush, reps=3):
    """The paper's GPU versions (Sec. IV-B to IV-E) beside the main path: one
    force evaluation of the 2^20-cell lattice whose rows come in a seeded random
    order (the order agents were created in, not a spatial one).  Each version's
    whole call (grid + forces) and the main path's grid build + force sweep."""
    import torch

    from paper_2105_00039_gb300 import populations as P
    from paper_2105_00039_gb300 import ugmech as U
    st = P.lattice_1m(0)
    n = len(st)
    order = np.argsort(P.uniform01(7, 301, n), kind="stable")
    x = torch.from_numpy(np.ascontiguousarray(st[order])).to(dev)
    prm = U.Params()
    lib = U.load()
    mb = U.estimate_max_boxes(x, 0.0)
    status = U.new_status(dev)
    out = {"workload": "2^20-cell lattice (102^3 sites, spacing 9), rows in a seeded random order; "
                       "one force evaluation including the grid"}
    ws = U.workspace(lib.ug_ladder_workspace_bytes(n, mb), dev)
    force = torch.empty((n, 4), dtype=torch.float64, device=dev)
    names = ("version0_fp64_lists", "version1_fp32_lists", "version2_fp32_sorted_lists",
             "version3_fp32_shared_atomics")
    for v, name in enumerate(names):
        def run(v=v):
            U._check(lib.ug_forces_ladder(v, U._ptr(x), n, prm.c(), mb, U._ptr(force), U._ptr(ws),
                                          ws.numel(), U._ptr(status), U._stream()), "ug_forces_ladder")
        run()
        U.check_status(status, "ug_forces_ladder")
        ms = _timed(run, reps, flush)
        U.check_status(status, "ug_forces_ladder")
        out[name] = {"ms": ms, "agents_per_s": n / (ms / 1e3)}
    del ws, force
    srt = torch.empty_like(x)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    start = torch.empty(mb + 1, dtype=torch.int32, device=dev)
    info = torch.empty(48, dtype=torch.uint8, device=dev)
    ws = U.workspace(lib.ug_workspace_bytes(n, 1, mb), dev)
    F = torch.empty_like(x)

    def main():
        U._check(lib.ug_grid_build(U._ptr(x), None, n, 0.0, U._ptr(srt), U._ptr(perm), U._ptr(start),
                                   mb, U._ptr(info), U._ptr(ws), ws.numel(), U._ptr(status),
                                   U._stream()), "ug_grid_build")
        U._check(lib.ug_compute_forces(U._ptr(srt), U._ptr(start), U._ptr(info), n, prm.c(), U._ptr(F),
                                       U._ptr(status), U._stream()), "ug_compute_forces")
    main()
    U.check_status(status, "main path")
    ms = _timed(main, reps, flush)
    U.check_status(status, "main path")
    out["main_path_grid_build_plus_forces"] = {"ms": ms, "agents_per_s": n / (ms / 1e3)}
    return out


def main():
    args = parse()
    world, rank, local, pg = dist_setup(args)
    try:
        if args.impl == "reference":
            run_reference(args, world, rank, pg)
        else:
            run_ours(args, world, rank, local, pg)
    finally:
        if pg is not None:
            pg.destroy_process_group()


if __name__ == "__main__":
    main()
