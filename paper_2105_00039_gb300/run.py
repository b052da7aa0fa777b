"""Step one seeded population on the GPU from the command line.

    python -m paper_2105_00039_gb300.run --cells 4194304 --neighbours 8 --steps 3 [--walk full|windows]

Builds the Benchmark-B style density cube (`populations.density_cube`, seed =
the neighbour count) or, with --lattice, the jittered lattice of the given
number of cells per axis, steps it with the fused step (maximum displacement
0 for the cube, as in the paper's benchmark B; the default constants for the
lattice) and prints the device time per step.  --walk picks the neighbour
walk of one simulation through `ug_step_batched` (full runs or windows);
without it `ug_step` chooses.  Useful as the workload of a profiler run.
"""
from __future__ import annotations

import argparse

import torch

from . import populations as P
from . import ugmech as U


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--cells", type=int, default=1 << 22)
    ap.add_argument("--neighbours", type=float, default=8.0)
    ap.add_argument("--lattice", type=int, default=0, help="cells per axis of a jittered lattice")
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--reps", type=int, default=1, help="timed repetitions after one untimed run")
    ap.add_argument("--walk", choices=["auto", "full", "windows"], default="auto")
    a = ap.parse_args(argv)
    dev = torch.device("cuda")
    if a.lattice:
        st = P.lattice_cube(a.lattice, seed=0)
        prm = U.Params()
    else:
        st = P.density_cube(a.cells, a.neighbours, seed=int(a.neighbours))
        prm = U.Params(max_disp=0.0)
    x0 = torch.from_numpy(st).to(dev)
    n = x0.shape[0]
    sp = U.Stepper(n, U.estimate_max_boxes(x0, prm.contact_margin, slack=1.05), dev)
    x = torch.empty_like(x0)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    one = torch.tensor([0, n], dtype=torch.int32, device=dev)
    tune = U.ug_tuning()
    tune.agents_per_lane, tune.sweep_block = 2, 128
    tune.neighbour_walk = {"full": 1, "windows": 2}.get(a.walk, 0)

    def run():
        x.copy_(x0)
        perm.copy_(torch.arange(n, dtype=torch.int32, device=dev))
        if a.walk == "auto":
            sp.step(x, perm, prm, a.steps)
        else:
            sp.step_batched(x, perm, one, prm.as_tensor(dev)[None], a.steps, tune)

    run()
    sp.check("run")
    for _ in range(a.reps):
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        run()
        t1.record()
        t1.synchronize()
        print(f"{n} cells: {1000.0 * t0.elapsed_time(t1) / a.steps:.1f} us per step", flush=True)
    sp.check("run")


if __name__ == "__main__":
    main()
