"""FP64 CPU oracle of the mechanical-interaction step (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and reference
legs may import this package.  It shares no code with the CUDA library.
"""
from .mech import (Params, grid, sub_bin_shift, pairs_bruteforce, pairs_kdtree, find_pairs, pair_terms,
                   forces, mass, displacement, step, trajectory, trajectory_grad,
                   trajectory_loss, mse_loss, margins, step_sampled,
                   trajectory_grad_along)

__all__ = ["Params", "grid", "sub_bin_shift", "pairs_bruteforce", "pairs_kdtree", "find_pairs", "pair_terms",
           "forces", "mass", "displacement", "step", "trajectory", "trajectory_grad",
           "trajectory_loss", "mse_loss", "margins", "step_sampled",
           "trajectory_grad_along"]
