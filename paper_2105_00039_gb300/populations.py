"""Seeded synthetic cell populations (inputs only; no mechanics here).

Every value is a pure function of (seed, stream, index) through a counter-based
SplitMix64 hash, so a population can be regenerated bit-for-bit anywhere.  The
shapes follow the workloads of Hesam et al. (Sec. III: a 3D grid of equal cells;
Sec. V, benchmark B: agents at random positions in a cube whose size sets the
mean neighbour count).  State layout is the library's: float32 rows
(x, y, z, diameter).

This module is shared by the CUDA path's callers and by the oracle's tests; it
holds no part of the force law, the grid or the integration.
"""
from __future__ import annotations

import math

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def _splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014) on uint64 counters."""
    with np.errstate(over="ignore"):
        z = x + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """n float64 uniforms in [0, 1) for counters start..start+n-1 of (seed, stream)."""
    with np.errstate(over="ignore"):
        base = _splitmix64(np.array([(seed * 0x100000001B3 + stream * 0x2545F4914F6CDD1D)
                                     & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
        ctr = np.arange(start, start + n, dtype=np.uint64) * _GOLDEN + base
    bits = _splitmix64(ctr) >> np.uint64(11)           # 53 random bits
    return bits.astype(np.float64) * (1.0 / 9007199254740992.0)


def _diameters(seed: int, n: int, dmin: float, dmax: float) -> np.ndarray:
    return dmin + (dmax - dmin) * uniform01(seed, 3, n)


def uniform_cube(n: int, side: float, dmin: float = 8.0, dmax: float = 12.0,
                 seed: int = 0) -> np.ndarray:
    """Centres uniform in [0, side]^3, diameters uniform in [dmin, dmax]."""
    out = np.empty((n, 4), dtype=np.float32)
    for a in range(3):
        out[:, a] = side * uniform01(seed, a, n)
    out[:, 3] = _diameters(seed, n, dmin, dmax)
    return out


def jittered_lattice(n: int, sites_per_axis: int, spacing: float, jitter: float,
                     dmin: float, dmax: float, seed: int = 0) -> np.ndarray:
    """The first n sites of a sites_per_axis^3 cubic lattice (x fastest, then y, z),
    each displaced by a uniform offset in [-jitter, jitter] per axis."""
    if n > sites_per_axis ** 3:
        raise ValueError("lattice has fewer sites than agents")
    idx = np.arange(n, dtype=np.int64)
    site = np.stack([idx % sites_per_axis, (idx // sites_per_axis) % sites_per_axis,
                     idx // (sites_per_axis * sites_per_axis)], axis=1).astype(np.float64)
    out = np.empty((n, 4), dtype=np.float32)
    for a in range(3):
        out[:, a] = spacing * site[:, a] + jitter * (2.0 * uniform01(seed, a, n) - 1.0)
    out[:, 3] = _diameters(seed, n, dmin, dmax)
    return out


def mean_cube_contact_volume(dmin: float, dmax: float) -> float:
    """(4 pi / 3) E[s^3] for s = (d1 + d2) / 2 with d ~ U[dmin, dmax] i.i.d.

    s = c + t with c the mid diameter and t the mean of two uniforms on
    [-w/2, w/2] (w = dmax - dmin), so E[s^3] = c^3 + 3 c Var(t) with
    Var(t) = w^2 / 24.  For d ~ U[8, 12] this is 1020.
    """
    c = 0.5 * (dmin + dmax)
    w = dmax - dmin
    return 4.0 * math.pi / 3.0 * (c ** 3 + 3.0 * c * w * w / 24.0)


def cube_side_for_neighbours(n: int, mean_neighbours: float, dmin: float = 8.0,
                             dmax: float = 12.0) -> float:
    """Cube side L giving an expected mean of `mean_neighbours` overlapping
    neighbours per agent for n uniform centres (ignoring the boundary)."""
    return (n * mean_cube_contact_volume(dmin, dmax) / mean_neighbours) ** (1.0 / 3.0)


def density_cube(n: int, mean_neighbours: float, dmin: float = 8.0, dmax: float = 12.0,
                 seed: int = 0) -> np.ndarray:
    """Benchmark-B style population: uniform centres in a cube sized for a target
    mean neighbour count."""
    return uniform_cube(n, cube_side_for_neighbours(n, mean_neighbours, dmin, dmax),
                        dmin, dmax, seed)


# ---------------------------------------------------------------- named workloads
def small_uniform(seed: int = 0) -> np.ndarray:
    """4,096 cells, centres uniform in a cube of side 160, diameters U[8, 12]."""
    return uniform_cube(4096, 160.0, 8.0, 12.0, seed)


def lattice_1m(seed: int = 0) -> np.ndarray:
    """2^20 cells: first 2^20 sites of a 102^3 lattice, spacing 9, jitter +-1.5,
    diameters U[9, 11]."""
    return jittered_lattice(1 << 20, 102, 9.0, 1.5, 9.0, 11.0, seed)


def lattice_cube(sites_per_axis: int, seed: int = 0) -> np.ndarray:
    """A full sites_per_axis^3 lattice with the same spacing/jitter/diameters as
    lattice_1m (64^3 = 262,144 is the differentiable workload)."""
    return jittered_lattice(sites_per_axis ** 3, sites_per_axis, 9.0, 1.5, 9.0, 11.0, seed)


def batched_population(nsims: int = 256, nmin: int = 1000, nmax: int = 200_000,
                       nb_lo: float = 4.0, nb_hi: float = 40.0, seed: int = 0,
                       dmin: float = 8.0, dmax: float = 12.0):
    """Many independent simulations of uneven size and density.

    Agent counts are log-uniform in [nmin, nmax], target mean neighbour counts
    uniform in [nb_lo, nb_hi].  Returns (state, sim_offset) with the sims'
    agents concatenated and sim_offset of length nsims + 1.
    """
    u = uniform01(seed, 101, nsims)
    counts = np.floor(np.exp(math.log(nmin) + (math.log(nmax) - math.log(nmin)) * u)).astype(np.int64)
    counts = np.clip(counts, nmin, nmax)
    nbar = nb_lo + (nb_hi - nb_lo) * uniform01(seed, 102, nsims)
    parts = [density_cube(int(c), float(nb), dmin, dmax, seed=seed * 1000003 + 7 + s)
             for s, (c, nb) in enumerate(zip(counts, nbar))]
    offs = np.zeros(nsims + 1, dtype=np.uint32)
    offs[1:] = np.cumsum(counts)
    return np.concatenate(parts, axis=0), offs


def random_unit_vectors(n: int, seed: int) -> np.ndarray:
    """One random direction over n agents' positions: an (n, 3) float64 array of
    unit (Frobenius) norm, for directional-derivative checks."""
    g = np.stack([uniform01(seed, 201 + a, n) for a in range(3)], axis=1) * 2.0 - 1.0
    g /= np.linalg.norm(g)
    return g
