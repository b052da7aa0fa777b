"""The paper's GPU versions (Sec. IV-B to IV-E) through ug_forces_ladder.

Version 0 evaluates Eq. 1 directly in float64, so it must find exactly the
oracle's overlapping pairs and agree with its forces to rounding.  Versions 1-3
evaluate the same formula in float32; for them the bound follows from float32
rounding (u = 2^-24): the difference of two rows is rounded relative to its
result, so d, and delta = r_i + r_j + 2m - d, are accurate to
ddelta = 8 u s (s = r_i + r_j + 2m), and Eq. 1 then moves by at most
kappa ddelta + gamma sqrt(R ddelta) per pair, plus relative rounding of the
products and sums (16 u of the pair's magnitude).  Pairs closer to touching
than ddelta may be found or missed.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2105_00039_gb300 import populations as P

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


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


def _reference(st, margin):
    prm = O.Params(contact_margin=margin)
    pos, diam = st[:, :3].astype(np.float64), st[:, 3].astype(np.float64)
    I, J = O.pairs_bruteforce(pos, 0.5 * diam, margin)
    F, S, npairs, t = O.forces(pos, diam, prm.as64(), I, J)
    s = 0.5 * diam[I] + 0.5 * diam[J] + 2.0 * margin
    dd = 8.0 * U32 * s
    mag = prm.k * t["delta"] + prm.gamma * t["root"]
    bound = np.bincount(I, weights=prm.k * dd + prm.gamma * np.sqrt(t["R"] * dd) + 16.0 * U32 * mag,
                        minlength=len(st))
    # pairs within ddelta of touching, on either side (a widened search finds the near misses)
    dmax = float(dd.max()) if len(dd) else 16.0 * U32 * float(diam.max())
    I2, J2 = O.pairs_bruteforce(pos, 0.5 * diam, margin + dmax)
    t2 = O.pair_terms(pos, diam, prm.as64(), I2, J2)
    s2 = 0.5 * diam[I2] + 0.5 * diam[J2] + 2.0 * margin
    delta2 = s2 - t2["d"]
    near = np.abs(delta2) <= 8.0 * U32 * s2
    r2 = 0.5 * diam
    R2 = r2[I2] * r2[J2] / (r2[I2] + r2[J2])
    dd2 = 8.0 * U32 * s2
    bound += np.bincount(I2[near & (delta2 <= 0)],
                         weights=(prm.k * dd2 + prm.gamma * np.sqrt(R2 * dd2))[near & (delta2 <= 0)],
                         minlength=len(st))
    return F, S, npairs, bound, np.bincount(I2[near], minlength=len(st))


@pytest.mark.parametrize("name", list(workloads()))
def test_version0_float64_matches_the_oracle(U, name):
    st, margin = workloads()[name]
    F, S, npairs, _, _ = _reference(st, margin)
    out = U.forces_ladder(torch.from_numpy(st).cuda(), 0, U.Params(contact_margin=margin)).cpu().numpy()
    assert np.array_equal(out[:, 3].astype(np.int64), npairs)
    err = np.abs(out[:, :3] - F).max(axis=1)
    assert (err <= 1e-9 * (1.0 + S)).all(), float((err / (1.0 + S)).max())


@pytest.mark.parametrize("version", [1, 2, 3])
@pytest.mark.parametrize("name", list(workloads()))
def test_float32_versions_within_rounding_bound(U, name, version):
    st, margin = workloads()[name]
    F, S, npairs, bound, near = _reference(st, margin)
    out = U.forces_ladder(torch.from_numpy(st).cuda(), version,
                          U.Params(contact_margin=margin)).cpu().numpy()
    assert (np.abs(out[:, 3].astype(np.int64) - npairs) <= near).all()
    err = np.abs(out[:, :3] - F).max(axis=1)
    assert (err <= bound + 1e-12).all(), float(np.max(err - bound))


def test_float32_versions_agree_with_each_other(U):
    st, margin = workloads()["dense_cube"]
    x = torch.from_numpy(st).cuda()
    outs = [U.forces_ladder(x, v, U.Params()).cpu().numpy() for v in (1, 2, 3)]
    F, S, npairs, bound, near = _reference(st, margin)
    for o in outs[1:]:
        assert np.array_equal(o[:, 3], outs[0][:, 3])
        assert (np.abs(o[:, :3] - outs[0][:, :3]).max(axis=1) <= 1e-5 * (1.0 + S)).all()


def test_version3_reports_an_overfull_neighbourhood(U):
    st = P.uniform_cube(1100, 4.0, 8.0, 12.0, 5)     # every agent in one box: 1100 > 1024 rows
    x = torch.from_numpy(st).cuda()
    with pytest.raises(U.UgError) as e:
        U.forces_ladder(x, 3, U.Params())
    assert e.value.code == U.UG_ECAPACITY
    out = U.forces_ladder(x, 2, U.Params())           # the list versions have no such limit
    assert int(out[:, 3].min().item()) == 1099
