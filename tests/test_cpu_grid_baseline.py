"""The CPU uniform-grid timing baseline (baseline/cpu_ug) computes the same
step as the FP64 oracle: positions after one step agree to the float32
rounding of its output rows, pair for pair on populations with and without a
contact margin, and over several steps."""
import os
import shutil
import sys

import numpy as np
import pytest

import oracle as O
from paper_2105_00039_gb300 import populations as P

sys.path.insert(0, os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                "baseline", "cpu_ug"))

pytestmark = pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")


def _ulp32(x):
    x = np.abs(np.asarray(x, dtype=np.float32))
    return (np.nextafter(x, np.float32(np.inf)) - x).astype(np.float64)


@pytest.mark.parametrize("case", ["uniform", "lattice_margin", "frozen"])
def test_one_step_matches_the_oracle(case):
    import cpu_ug
    if case == "uniform":
        st, kw = P.small_uniform(0), {}
    elif case == "lattice_margin":
        st, kw = P.jittered_lattice(4096, 16, 9.0, 1.5, 9.0, 11.0, 1), {"contact_margin": 1.5}
    else:
        st, kw = P.uniform_cube(3000, 60.0, 8.0, 12.0, 2), {"max_disp": 0.0}
    out, secs = cpu_ug.steps(st, 1, threads=2, **kw)
    ref = O.step(st, O.Params(**kw))
    assert secs > 0.0
    err = np.abs(out[:, :3].astype(np.float64) - ref["state"][:, :3])
    assert (err <= _ulp32(ref["state"][:, :3])).all()
    if case == "frozen":
        assert np.array_equal(out, st)


def test_three_steps_track_the_oracle():
    import cpu_ug
    st = P.small_uniform(3)
    out, _ = cpu_ug.steps(st, 3, threads=3, adherence=0.0)
    ref = O.trajectory(st, O.Params(adherence=0.0), nsteps=3)
    assert np.abs(out[:, :3].astype(np.float64) - ref[:, :3]).max() < 1e-3
