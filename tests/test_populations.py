"""Pins for the seeded input generators (CPU): the counter-based hash against
the published SplitMix64 sequence, the uniforms' range and moments, the lattice
layout, the closed form behind the density cubes (checked by sampling and by
counting contacts away from the faces), and the batched population's
structure."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2105_00039_gb300 import populations as P

GOLDEN = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1


def test_splitmix64_matches_the_published_sequence():
    # SplitMix64 (Steele, Lea, Flood 2014) seeded with 0 adds the golden gamma
    # to its state before each output; its first three outputs are
    # 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f.  The
    # generator's finaliser applied to the states k * gamma reproduces them.
    states = np.array([(k * GOLDEN) & M64 for k in range(3)], dtype=np.uint64)
    out = [int(v) for v in P._splitmix64(states)]
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniforms_range_moments_and_counters():
    n = 1 << 20
    u = P.uniform01(7, 0, n)
    assert u.dtype == np.float64 and u.min() >= 0.0 and u.max() < 1.0
    se = math.sqrt(1.0 / 12.0 / n)
    assert abs(u.mean() - 0.5) < 6 * se
    assert abs(u.var() - 1.0 / 12.0) < 6 * math.sqrt(1.0 / 180.0 / n)
    v = P.uniform01(7, 1, n)                                  # another stream
    assert abs(np.corrcoef(u, v)[0, 1]) < 6 / math.sqrt(n)
    assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 6 / math.sqrt(n)   # successive counters
    np.testing.assert_array_equal(P.uniform01(7, 0, 10, start=5), u[5:15])
    np.testing.assert_array_equal(P.uniform01(7, 0, 1000), u[:1000])  # pure function
    assert not np.array_equal(P.uniform01(8, 0, 1000), u[:1000])


def test_lattice_layout_and_jitter():
    st = P.jittered_lattice(8, 2, 9.0, 0.0, 10.0, 10.0, 0)
    np.testing.assert_array_equal(st[:, :3], [[0, 0, 0], [9, 0, 0], [0, 9, 0], [9, 9, 0],
                                              [0, 0, 9], [9, 0, 9], [0, 9, 9], [9, 9, 9]])
    assert np.all(st[:, 3] == 10.0)
    st = P.jittered_lattice(1000, 10, 9.0, 1.5, 9.0, 11.0, 3)
    idx = np.arange(1000)
    site = 9.0 * np.stack([idx % 10, idx // 10 % 10, idx // 100], axis=1)
    off = st[:, :3].astype(np.float64) - site
    assert np.abs(off).max() <= 1.5 + 1e-5 and np.abs(off).max() > 1.4
    assert st[:, 3].min() >= 9.0 and st[:, 3].max() <= 11.0
    with pytest.raises(ValueError):
        P.jittered_lattice(9, 2, 9.0, 0.0, 10.0, 10.0, 0)


def test_lattice_1m_recipe():
    st = P.lattice_1m(0)
    assert st.shape == (1 << 20, 4) and st.dtype == np.float32
    # the first 2^20 sites of 102^3, x fastest: the last cell sits at site
    # (1048575 % 102, 1048575 // 102 % 102, 1048575 // 102^2) = (15, 80, 100)
    last = 9.0 * np.array([15, 80, 100])
    assert np.abs(st[-1, :3] - last).max() <= 1.5 + 1e-4
    assert st[:, 3].min() >= 9.0 and st[:, 3].max() <= 11.0


def test_contact_volume_closed_form():
    # s = (d1 + d2) / 2, d ~ U[8, 12]: E[s^3] = 10^3 + 3 * 10 * Var(s), Var(s) = 16/24
    assert abs(P.mean_cube_contact_volume(8.0, 12.0) - 4.0 * math.pi / 3.0 * 1020.0) < 1e-9
    d = np.random.default_rng(0).uniform(8.0, 12.0, size=(2, 2_000_000))
    mc = float(np.mean((0.5 * (d[0] + d[1])) ** 3))
    assert abs(mc - 1020.0) < 1.0
    L = P.cube_side_for_neighbours(4 << 20, 8.0)
    assert abs(L - 1308.4) < 0.1                              # the 4M-cell, 8-neighbour cube


@pytest.mark.parametrize("nbar,tol", [(8.0, 0.15), (32.0, 0.4)])
def test_density_cube_gives_its_mean_neighbours_away_from_the_faces(nbar, tol):
    """Cells farther than the largest contact distance from every face have
    the target mean number of overlapping neighbours (contacts by the oracle's
    exact pair search)."""
    n = 30000
    st = P.density_cube(n, nbar, seed=5).astype(np.float64)
    L = P.cube_side_for_neighbours(n, nbar)
    I, _ = O.pairs_kdtree(st[:, :3], 0.5 * st[:, 3])
    cnt = np.bincount(I, minlength=n)
    inner = np.all((st[:, :3] > 12.0) & (st[:, :3] < L - 12.0), axis=1)
    assert inner.sum() > n // 2
    assert abs(cnt[inner].mean() - nbar) < tol


def test_batched_population_structure():
    st, offs = P.batched_population(nsims=16, nmin=1000, nmax=20000, seed=2)
    counts = np.diff(offs.astype(np.int64))
    assert offs[0] == 0 and offs[-1] == len(st) and len(offs) == 17
    assert counts.min() >= 1000 and counts.max() <= 20000
    assert st.dtype == np.float32 and st[:, 3].min() >= 8.0 and st[:, 3].max() <= 12.0
    again, offs2 = P.batched_population(nsims=16, nmin=1000, nmax=20000, seed=2)
    assert np.array_equal(st, again) and np.array_equal(offs, offs2)


def test_random_direction_has_unit_norm():
    v = P.random_unit_vectors(500, seed=4)
    assert v.shape == (500, 3) and abs(np.linalg.norm(v) - 1.0) < 1e-12
