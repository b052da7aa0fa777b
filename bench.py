#!/usr/bin/env python
"""Throughput of the mechanical-interaction step (agent-steps/s).

Workload: 2^20 cells on a jittered 102^3 lattice (spacing 9, jitter +-1.5,
diameters U[9, 11]), 100 fused steps with the grid rebuilt every step.  One
bench step = those 100 steps from the same initial rows, so a bench step
processes 2^20 * 100 agent-steps.  Before each timed step a 256 MB buffer is
written to flush the 129 MB L2 (outside the step's CUDA events).

Prints one JSON line (rank 0).  --impl reference times the FP64 oracle on the
host cores on a bounded sample of the same workload instead.

Multi-GPU: the path is weak-scaled as independent replicas (each rank runs its
own population; no collective on the data path); the barrier and the max over
ranks only frame the timing.
"""
import argparse
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

N_LATTICE = 1 << 20
SIM_STEPS = 100
BYTES_PER_AGENT_SWEEP = 32          # sweep + move: read 16 B row, write 16 B row
BYTES_PER_AGENT_STEP = 88           # whole step (grid bin 16, scatter 40, sweep 32)
BYTES_PER_BOX = 12
# algorithmic FP32 operations: distance pre-test per candidate pair (3 sub,
# 3 mul/fma, 1 add, 1 mul, 1 compare), Eq. 1 per contact (delta: sqrt + sub; R:
# mul, add, div; sqrt(R delta): mul + sqrt; phi: 2 mul + sub; direction: div +
# 3 mul; sum: 3 add) and the displacement per agent (|F|, mass, dt/m, 3 mul,
# |v|, cap test, 3 add)
FLOPS_PER_CANDIDATE = 9
FLOPS_PER_CONTACT = 17
FLOPS_PER_AGENT = 25
# FP32 roof: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# DRAM bytes (read + write) of one k_sweep2 launch on this workload, from the
# ncu capture summarised in profiles/k_sweep2_lattice1m.md (cache flushed)
SWEEP_DRAM_BYTES = 23.521792e6 + 0.320256e6
SWEEP_DRAM_BYTES_SRC = "9b362eb61c0f7119"      # sha256[:16] of ug_sweep2.cu + ug_internal.cuh when captured


# Warp instructions of one k_sweep2 launch on this workload, from the same ncu
# capture (and valid under the same source check) as the DRAM bytes above, and
# the SMs' issue limit: one warp instruction per scheduler per clock, four
# schedulers per SM.
SWEEP_WARP_INST = 89_700_118
ISSUE_PEAK_GINST_S = 152 * 4 * 2.07


def issue_roofline(avg_launch_ms: float):
    """The sweep against the instruction-issue limit (the bound that holds it),
    or None once its source has changed since the instruction count was taken."""
    if sweep_traffic() is None:
        return None
    achieved = SWEEP_WARP_INST / (avg_launch_ms / 1000.0) / 1e9
    return {"warp_inst_per_launch": SWEEP_WARP_INST, "achieved_ginst_s": achieved,
            "peak_ginst_s": ISSUE_PEAK_GINST_S, "frac": achieved / ISSUE_PEAK_GINST_S,
            "peak_source": "derived: 152 SMs x 4 schedulers x 1 warp instruction per clock "
                           "x 2.07 GHz; instructions per launch from ncu"}


def sweep_traffic():
    """The captured DRAM bytes if the sweep's source is unchanged since, else None."""
    import hashlib
    h = hashlib.sha256()
    for f in ("ug_sweep2.cu", "ug_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2105_00039_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return SWEEP_DRAM_BYTES if h.hexdigest()[:16] == SWEEP_DRAM_BYTES_SRC else None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched, adjoint and density-sweep rows")
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


def cpu_oracle_rate(state, nsteps_sample: int):
    """The FP64 oracle as it stands, one full step of the whole population per
    sample step; returns (agent-steps/s, seconds)."""
    import oracle as O
    t0 = time.perf_counter()
    st = state
    for _ in range(nsteps_sample):
        st = O.step(st, O.Params())["state"]
    dt = time.perf_counter() - t0
    return len(state) * nsteps_sample / dt, dt


def candidates_and_contacts(U, x, prm):
    """Mean candidates (agents in the 27 surrounding boxes, self excluded) and
    contacts per agent of a population, from the library's grid and forces.
    Measurement only: the box counts are summed over 3x3x3 neighbourhoods with
    torch on the box table."""
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
    return cand, float(F[:, 3].double().mean().item())


def run_reference(args, world, rank, pg):
    from paper_2105_00039_gb300 import populations as P
    if rank != 0:
        return
    st = P.lattice_1m(0)
    for _ in range(args.warmup):
        cpu_oracle_rate(st, 1)
    times = []
    for _ in range(args.steps):
        _, dt = cpu_oracle_rate(st, 1)
        times.append(dt)
    total = sum(times)
    value = len(st) * args.steps / total
    line = {
        "impl": "reference", "metric": "agent-steps/s", "value": value, "unit": "agent-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "lattice_1m: 2^20 cells, 102^3 lattice spacing 9 jitter 1.5, d U[9,11]",
                   "n_agents": len(st), "sample": "1 oracle step of the full population per bench step",
                   "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "agent-steps/s", "cores": 1, "kind": "oracle",
                         "sample": "1 FP64 oracle step (cKDTree pair search + numpy Eq. 1) of all 2^20 cells per bench step"},
        "e2e": {"value": value, "unit": "agent-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local, pg):
    import torch

    from paper_2105_00039_gb300 import populations as P
    from paper_2105_00039_gb300 import ugmech as U

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    st = P.lattice_1m(seed=rank)
    n = len(st)
    prm = U.Params()
    x0 = torch.from_numpy(st).to(dev)
    x = torch.empty_like(x0)
    max_boxes = U.estimate_max_boxes(x0, prm.contact_margin, slack=1.5)
    sp = U.Stepper(n, max_boxes, dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    nev = 2 + 5 * SIM_STEPS
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    lib = U.load()
    stream = torch.cuda.current_stream()

    def reset():
        x.copy_(x0)
        U._check(lib.ug_iota(U._ptr(perm), n, U._stream()), "ug_iota")

    # warm-up (also creates the CUDA handles of the trace events)
    events = [torch.cuda.Event(enable_timing=True) for _ in range(nev)]
    for e in events:
        e.record(stream)
    for _ in range(args.warmup):
        reset()
        sp.step(x, perm, prm, SIM_STEPS)
    sp.check("warm-up")
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kern_ms = {k: 0.0 for k in ("bounds", "key", "scan", "place", "canon", "sweep")}
    names = ["key", "scan", "place", "canon", "sweep"]
    if pg is not None:
        pg.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        # the metric: K plain bench steps (kernels chained with programmatic
        # dependent launch), each preceded by an L2 flush outside its events
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            reset()
            sp.step(x, perm, prm, SIM_STEPS)
            ends[k].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        # per-kernel durations: the same K bench steps again with CUDA events
        # recorded between the kernels (which also un-chains them)
        for k in range(args.steps):
            flush.zero_()
            reset()
            sp.step_traced(x, perm, prm, SIM_STEPS, events)
            events[-1].synchronize()
            kern_ms["bounds"] += events[0].elapsed_time(events[1])
            for t in range(SIM_STEPS):
                for j, nm in enumerate(names):
                    kern_ms[nm] += events[1 + 5 * t + j].elapsed_time(events[2 + 5 * t + j])
        torch.cuda.synchronize()
    if pg is not None:
        pg.barrier()
    sp.check("timed steps")
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    tot_ms = reduce_max(pg, sum(step_ms), dev)
    ms_per_step = tot_ms / args.steps
    value = world * n * SIM_STEPS * args.steps / (tot_ms / 1000.0)

    # roofline of the dominant kernel (time-weighted, per launch)
    launches = {"bounds": args.steps, **{nm: args.steps * SIM_STEPS for nm in names}}
    dom = max(kern_ms, key=kern_ms.get)
    avg_launch_ms = kern_ms[dom] / launches[dom]
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        peaks = json.load(f)
    hbm = float(peaks["hbm_gbs"])
    alg_bytes = {"sweep": BYTES_PER_AGENT_SWEEP * n, "canon": 48 * n, "key": 24 * n,
                 "place": 16 * n, "scan": 12 * max_boxes, "bounds": 16 * n}[dom]
    achieved = alg_bytes / (avg_launch_ms / 1000.0) / 1e9
    # candidates and contacts at the start and the end of a bench step
    c0, k0 = candidates_and_contacts(U, x0, prm)
    c1, k1 = candidates_and_contacts(U, x.contiguous(), prm)
    cand, cont = 0.5 * (c0 + c1), 0.5 * (k0 + k1)
    alg_flops = n * (FLOPS_PER_CANDIDATE * cand + FLOPS_PER_CONTACT * cont + FLOPS_PER_AGENT)
    alu_tflops = alg_flops / (avg_launch_ms / 1000.0) / 1e12
    # whole-step HBM roofline (algorithmic bytes of the method per step)
    step_alg = (BYTES_PER_AGENT_STEP * n + BYTES_PER_BOX * max_boxes / 1.5) * SIM_STEPS
    step_gbs = step_alg / (ms_per_step / 1000.0) / 1e9

    line = {
        "metric": "agent-steps/s", "value": value, "unit": "agent-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "lattice_1m: 2^20 cells, 102^3 lattice spacing 9 jitter 1.5, d U[9,11]; "
                               "100 fused steps (grid rebuilt each step) per bench step",
                   "n_agents": n, "sim_steps_per_step": SIM_STEPS, "max_boxes": max_boxes,
                   "l2": "flushed (256 MB write) before each timed step, outside its events",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "alu", "kernel": dom, "achieved": alu_tflops,
                     "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": alu_tflops / FP32_PEAK_TFLOPS,
                     "traffic": sweep_traffic() if dom == "sweep" else None,
                     "avg_launch_us": avg_launch_ms * 1000.0,
                     "alg_flops_per_launch": alg_flops,
                     "candidates_per_agent": cand, "contacts_per_agent": cont,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                     "note": "instruction issue: 68% of issue slots busy, 89.7M warp instructions per launch (ncu), see profiles/k_sweep2_lattice1m.md",
                     "issue": issue_roofline(avg_launch_ms) if dom == "sweep" else None,
                     "hbm": {"achieved_gbs": achieved, "peak_gbs": hbm, "frac": achieved / hbm,
                             "alg_bytes_per_launch": alg_bytes,
                             "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"},
                     "step_alg_gbs": step_gbs, "step_hbm_frac": step_gbs / hbm},
        "kernel_ms_share": {k: v / sum(kern_ms.values()) for k, v in kern_ms.items()},
        "gpu_launches": args.steps * (2 + 5 * SIM_STEPS),
        "kernel_ms_per_step_traced": {k: v / (args.steps * SIM_STEPS) for k, v in kern_ms.items()},
        "clocks": clk.summary(),
        "wall_s_timed_region": wall,
    }

    # end to end through the public API: pinned host rows in, rows (by id) out
    if not args.no_e2e:
        sim = U.Simulation(n, max_boxes, dev)
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

    # the extra rows and the CPU baselines are single-GPU measurements: a
    # multi-GPU run reports only the headline
    if not args.no_extras and world == 1:
        line["batched"] = measure_batched(dev, flush)
        line["adjoint"] = measure_adjoint(dev, flush)
        line["density_sweep"] = measure_density(dev, flush)
        line["version_ladder"] = measure_ladder(dev, flush)
        line["lattice_margin"] = measure_lattice_margin(dev, flush)
        line["pairs_once"] = measure_pairs_once(dev, flush)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, secs = cpu_oracle_rate(st, 6)
        line["cpu_baseline"] = {"value": rate, "unit": "agent-steps/s", "cores": 1, "kind": "oracle",
                                "sample": f"6 FP64 oracle steps of all 2^20 cells ({secs:.1f} s)"}
        line["cpu_grid_baseline"] = cpu_grid_rate(st, 50)
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


def measure_batched(dev, flush, nsims=256, nsteps=50, reps=3):
    """256 independent simulations (agent counts log-uniform in [1e3, 2e5], mean
    neighbours U[4, 40]), 50 steps: the batched step captured as one CUDA graph
    versus the 256 simulations run one after another with the plain step of
    the same method (ug_step, or ug_step_pairs_once when the tuner picks every
    pair once)."""
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

    def batched():
        sp.step_batched(x, perm, offs_t, pdev, nsteps, tune)

    s = torch.cuda.Stream(device=dev)
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        reset()
        batched()                                  # warm-up outside capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            batched()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()

    def run_graph():
        reset()
        g.replay()
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
    return {"workload": f"{nsims} simulations, {n} agents in total, {nsteps} steps",
            "batched_graph_ms": t_batched, "sequential_plain_ms": t_seq,
            "batched_agent_steps_per_s": n * nsteps / (t_batched / 1e3),
            "sequential_agent_steps_per_s": n * nsteps / (t_seq / 1e3),
            "speedup": t_seq / t_batched, "bit_identical_to_plain": bool(same),
            "tuned_sweep_block": int(tune.sweep_block),
            "tuned_agents_per_lane": int(tune.agents_per_lane),
            "tuned_pair_mode": int(tune.pair_mode)}


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


def measure_lattice_margin(dev, flush, margin=1.5, nsteps=100, reps=2):
    """The headline lattice with each contact radius widened by a margin of 1.5
    (the variant that reaches ~12 overlapping neighbours per cell), 100 fused
    steps: agent-steps/s and the measured mean neighbour count."""
    import torch

    from paper_2105_00039_gb300 import populations as P
    from paper_2105_00039_gb300 import ugmech as U
    st = P.lattice_1m(0)
    n = len(st)
    x0 = torch.from_numpy(st).to(dev)
    prm = U.Params(contact_margin=margin)
    mb = U.estimate_max_boxes(x0, margin, slack=1.2)
    sp = U.Stepper(n, mb, dev)
    x = torch.empty_like(x0)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    lib = U.load()

    def run():
        x.copy_(x0)
        U._check(lib.ug_iota(U._ptr(perm), n, U._stream()), "ug_iota")
        sp.step(x, perm, prm, nsteps)
    run()
    sp.check("lattice margin")
    ms = _timed(run, reps, flush)
    sp.check("lattice margin")
    srt, _, start, info, _ = U.grid_build(x0, contact_margin=margin)
    F = U.compute_forces(srt, start, info, prm)
    return {"workload": f"lattice_1m with contact margin {margin}, {nsteps} fused steps",
            "agent_steps_per_s": n * nsteps / (ms / 1e3), "ms_per_step": ms / nsteps,
            "mean_neighbours_initial": float(F[:, 3].double().mean().item())}


def measure_pairs_once(dev, flush, reps=5):
    """Newton's third law (ug_forces_symmetric) on the box-sorted 2^20-cell
    lattice: one force evaluation with every pair evaluated once (forward half
    of each neighbourhood, fixed-point atomics to both agents), the same walk
    over all 27 boxes, and the main path's force sweep (ug_compute_forces)."""
    import torch

    from paper_2105_00039_gb300 import populations as P
    from paper_2105_00039_gb300 import ugmech as U
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


def measure_density(dev, flush, reps=2, nsteps=20):
    """Benchmark-B style density sweep: uniform centres in cubes sized for a mean
    of 2, 8, 32, 64 overlapping neighbours (4,194,304 cells) and 12 (16,777,216
    cells), max displacement 0 (frozen), 20 steps each, with ug_step and with
    ug_step_pairs_once."""
    import torch

    from paper_2105_00039_gb300 import populations as P
    from paper_2105_00039_gb300 import ugmech as U
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        hbm = float(json.load(f)["hbm_gbs"])
    prm = U.Params(max_disp=0.0)
    rows = []
    lib = U.load()
    for n, nbar in ((1 << 22, 2), (1 << 22, 8), (1 << 22, 32), (1 << 22, 64), (1 << 24, 12)):
        st = P.density_cube(n, float(nbar), seed=nbar)
        x0 = torch.from_numpy(st).to(dev)
        del st
        mb = U.estimate_max_boxes(x0, 0.0, slack=1.05)
        sp = U.Stepper(n, mb, dev)
        x = torch.empty_like(x0)
        perm = torch.empty(n, dtype=torch.int32, device=dev)

        def run(pairs_once=False):
            x.copy_(x0)
            U._check(lib.ug_iota(U._ptr(perm), n, U._stream()), "ug_iota")
            sp.step(x, perm, prm, nsteps, pairs_once=pairs_once)
        run(); sp.check("density"); torch.cuda.synchronize()
        ms = _timed(run, reps, flush)
        sp.check("density")
        # the same steps with every pair evaluated once (ug_step_pairs_once)
        run(True); sp.check("density, pairs once"); torch.cuda.synchronize()
        ms_once = _timed(lambda: run(True), reps, flush)
        sp.check("density, pairs once")
        per_step_s = ms / 1e3 / nsteps
        alg = BYTES_PER_AGENT_STEP * n + BYTES_PER_BOX * mb / 1.05
        # one traced pass for the per-kernel split (events un-chain the kernels)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 + 5 * nsteps)]
        for e in ev:
            e.record()
        x.copy_(x0)
        U._check(lib.ug_iota(U._ptr(perm), n, U._stream()), "ug_iota")
        sp.step_traced(x, perm, prm, nsteps, ev)
        ev[-1].synchronize()
        names = ("key", "scan", "place", "canon", "sweep")
        split = {nm: sum(ev[1 + 5 * t + j].elapsed_time(ev[2 + 5 * t + j]) for t in range(nsteps))
                 * 1000.0 / nsteps for j, nm in enumerate(names)}
        # the sweep against the FP32 ALU roof (the population is frozen: counts hold every step)
        cand, cont = candidates_and_contacts(U, x0, prm)
        flops = n * (FLOPS_PER_CANDIDATE * cand + FLOPS_PER_CONTACT * cont + FLOPS_PER_AGENT)
        tflops = flops / (split["sweep"] * 1e-6) / 1e12
        rows.append({"n_agents": n, "mean_neighbours_target": nbar,
                     "agent_steps_per_s": n * nsteps / (ms / 1e3), "ms_per_step": per_step_s * 1e3,
                     "step_alg_gbs": alg / per_step_s / 1e9, "step_hbm_frac": alg / per_step_s / 1e9 / hbm,
                     "pairs_once_agent_steps_per_s": n * nsteps / (ms_once / 1e3),
                     "pairs_once_ms_per_step": ms_once / nsteps,
                     "candidates_per_agent": cand, "contacts_per_agent": cont,
                     "sweep_alu_tflops": tflops, "sweep_alu_frac": tflops / FP32_PEAK_TFLOPS,
                     "kernel_us_per_step_traced": split})
        del x0, x, perm, sp
        torch.cuda.empty_cache()
    return rows


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
