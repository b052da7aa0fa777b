"""Symmetric (Newton's third law) pair evaluation through ug_forces_symmetric:
each overlapping pair evaluated once, its force added to both agents in 64-bit
fixed point.  Against the FP64 oracle within the per-step tolerance, pair
counts exact, the same bits as walking every pair from both sides, and
within float32 rounding of the main path's compensated sums."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2105_00039_gb300 import populations as P

from _metrics import TOL_STEP, by_id, force_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def U():
    from paper_2105_00039_gb300 import ugmech
    ugmech.load()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return ugmech


def workloads():
    return {
        "uniform4096": (P.small_uniform(0), 0.0),
        "lattice4096_margin": (P.jittered_lattice(4096, 16, 9.0, 1.5, 9.0, 11.0, 1), 1.5),
        "dense_cube": (P.uniform_cube(3000, 60.0, 8.0, 12.0, 2), 0.0),
        "ragged_777": (P.uniform_cube(777, 70.0, 8.0, 12.0, 3), 0.0),
    }


@pytest.mark.parametrize("name", list(workloads()))
def test_pairs_once_match_oracle_and_both_sides(U, name):
    st, margin = workloads()[name]
    prm_u = U.Params(contact_margin=margin)
    x = torch.from_numpy(st).cuda()
    srt, perm, start, info, _ = U.grid_build(x, contact_margin=margin)
    once = U.forces_symmetric(srt, start, info, prm_u, each_pair_once=True)
    both = U.forces_symmetric(srt, start, info, prm_u, each_pair_once=False)
    assert torch.equal(once, both)
    pid = perm.cpu().numpy()
    F = by_id(once.cpu().numpy().astype(np.float64), pid)
    prm = O.Params(contact_margin=margin).as64()
    pos, diam = st[:, :3].astype(np.float64), st[:, 3].astype(np.float64)
    I, J = O.pairs_bruteforce(pos, 0.5 * diam, margin)
    Fr, S, npairs, _ = O.forces(pos, diam, prm, I, J)
    assert np.array_equal(F[:, 3].astype(np.int64), npairs)
    per, norm, bad = force_errors(F[:, :3], Fr, S)
    assert per <= TOL_STEP and bad == 0, (per, bad)
    # and against the main path (compensated float32 sums): same pairs, forces
    # within float32 rounding of the per-agent scale
    main = U.compute_forces(srt, start, info, prm_u).cpu().numpy().astype(np.float64)
    assert np.array_equal(main[:, 3], once.cpu().numpy()[:, 3])
    Ss = S[pid]
    assert (np.abs(main[:, :3] - once.cpu().numpy()[:, :3]).max(axis=1) <= 1e-6 * (1.0 + Ss)).all()


def test_pairs_once_is_deterministic_on_a_large_population(U):
    st = P.density_cube(1 << 18, 20.0, seed=41)
    x = torch.from_numpy(st).cuda()
    srt, perm, start, info, _ = U.grid_build(x)
    a = U.forces_symmetric(srt, start, info, U.Params())
    b = U.forces_symmetric(srt, start, info, U.Params())
    c = U.forces_symmetric(srt, start, info, U.Params(), each_pair_once=False)
    assert torch.equal(a, b) and torch.equal(a, c)
    # Newton's third law: the forces of all agents sum to zero (fixed point: exactly)
    tot = a[:, :3].double().sum(0).abs().max().item()
    assert tot < 1e-2   # float32 rounding of each agent's fixed-point sum
