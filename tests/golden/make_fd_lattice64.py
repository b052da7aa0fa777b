"""Writes fd_lattice64.json: FP64 central differences of the differentiable
workload's loss, computed with the oracle alone.

Workload: 64^3 = 262,144 cells on the jittered lattice (spacing 9, jitter
+-1.5, diameters U[9, 11], seed 5), 50 steps with adherence 0, loss = mean over
coordinates of (p_50 - p^_50)^2 where p^ is the trajectory of the same start
with kappa = 2.5, gamma = 1.2.  Derivatives at kappa = 2, gamma = 1 (Eq. 1's
coefficients), by central differences at h = 3e-3, 1e-3 and 3e-4, beside the
oracle's own reverse-mode gradient along its FP64 trajectory.  The spread of the
differences over h shows the kinks that sqrt(delta) puts into the loss where a
pair starts or stops touching.

Run from the repository root:  python tests/golden/make_fd_lattice64.py
(about 15 minutes of one core per trajectory group; the differences run in a
spawned process pool).
"""
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

SIDE, SEED, STEPS = 64, 5, 50
HS = (3e-3, 1e-3, 3e-4)


_TARGET = None


def _init(target):
    global _TARGET
    _TARGET = target


def _loss(args):
    k, g = args
    import oracle as O
    from paper_2105_00039_gb300 import populations as P
    st = P.lattice_cube(SIDE, seed=SEED)
    return O.trajectory_loss(st, _TARGET, O.Params(k=k, gamma=g, adherence=0.0), STEPS, "kdtree")


def main():
    import oracle as O
    from paper_2105_00039_gb300 import populations as P
    t0 = time.time()
    st = P.lattice_cube(SIDE, seed=SEED)
    target = O.trajectory(st, O.Params(k=2.5, gamma=1.2, adherence=0.0), STEPS, "kdtree")[:, :3]
    jobs = []
    for h in HS:
        jobs += [(2.0 + h, 1.0), (2.0 - h, 1.0), (2.0, 1.0 + h), (2.0, 1.0 - h)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(jobs), os.cpu_count() or 1), initializer=_init, initargs=(target,)) as pool:
        vals = pool.map(_loss, jobs)
    fd = []
    for q, h in enumerate(HS):
        kp, km, gp, gm = vals[4 * q: 4 * q + 4]
        fd.append({"h": h, "dL_dkappa": (kp - km) / (2 * h), "dL_dgamma": (gp - gm) / (2 * h)})
    ref = O.trajectory_grad(st, target, O.Params(adherence=0.0), STEPS, "kdtree")
    out = {
        "workload": f"{SIDE}^3 jittered lattice (spacing 9, jitter 1.5, d U[9,11], seed {SEED}), "
                    f"{STEPS} steps, adherence 0; target from kappa 2.5, gamma 1.2",
        "at": {"kappa": 2.0, "gamma": 1.0},
        "loss": ref["loss"],
        "oracle_adjoint": {"dL_dkappa": ref["dk"], "dL_dgamma": ref["dgamma"]},
        "central_differences": fd,
        "seconds": round(time.time() - t0, 1),
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "fd_lattice64.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
