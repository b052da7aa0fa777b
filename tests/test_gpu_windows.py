"""The windowed neighbour walk against the full three-box runs.

The fused step cuts each neighbour row down to the x-window that can hold an
agent's contacts (sub-bins of the box table, the row's y/z gaps).  A window
that missed a contact would change the force sums, and an extra candidate is
rejected by the contact test, so the two walks must give the same bits: both
meet an agent's contacts in the same order.  Checked through the C ABI:
ug_step_batched with one simulation walks the full runs (neighbour_walk 1),
the windows at every number of x slices per box (2) or where they pay (0, as
ug_step does; the constants then come from device memory), and all must equal
ug_step
on populations whose grids use 1, 2, 4 and 8 x slices per box, at the edges of
the method (a slab a few boxes thick, agents on box faces, everything near the
origin, an odd agent count), and at full size.  The every-pair-once step walks
its forward rows through the same windows: its fixed-point sums do not depend
on the order, so windows and full runs must give the same bits there too, for
one simulation and for several.
"""
import numpy as np
import pytest
import torch

from paper_2105_00039_gb300 import populations as P

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def U():
    from paper_2105_00039_gb300 import ugmech
    ugmech.load()
    return ugmech


def _run(U, st, prm, nsteps, walk):
    x = torch.from_numpy(np.ascontiguousarray(st, np.float32)).to(DEV)
    n = x.shape[0]
    mb = U.estimate_max_boxes(x, prm.contact_margin, slack=2.0, extra_extent=8.0 * nsteps)
    sp = U.Stepper(n, mb, x.device)
    perm = U.iota(n, x.device)
    if walk == "step":
        sp.step(x, perm, prm, nsteps)
    else:                      # one simulation through the batched entry (constants on the device)
        offs = torch.tensor([0, n], dtype=torch.int32, device=DEV)
        t = U.ug_tuning()
        t.agents_per_lane, t.sweep_block = 2, 128
        t.neighbour_walk = {"batched_full_runs": 1, "batched_windows": 2, "batched_default": 0}[walk]
        sp.step_batched(x, perm, offs, prm.as_tensor(DEV)[None], nsteps, t)
    sp.check()
    return x, perm


def _same(U, st, prm, nsteps=3, ways=("step", "batched_full_runs", "batched_windows",
                                      "batched_default")):
    a, pa = _run(U, st, prm, nsteps, ways[0])
    for how in ways[1:]:
        b, pb = _run(U, st, prm, nsteps, how)
        assert torch.equal(pa, pb), how
        assert torch.equal(a, b), how
    return a


def _cases():
    face = P.jittered_lattice(3000, 15, 10.0, 0.0, 10.0, 10.0, 4).copy()   # centres on box faces
    face[:, :3] -= face[:, :3].min(axis=0)
    slab = P.uniform_cube(4000, 220.0, 8.0, 12.0, 6).copy()
    slab[:, 2] = 20.0 * slab[:, 2] / 220.0                                     # 3-4 boxes thick
    near = P.uniform_cube(3001, 40.0, 8.0, 12.0, 8).copy()
    near[:, :3] -= 20.0                                                        # around the origin
    return {
        "sparse_K1": (P.density_cube(20000, 2.0, seed=1), 0.0),
        "lattice_K2": (P.jittered_lattice(20000, 28, 7.0, 1.0, 9.0, 11.0, 2), 0.0),
        "dense_K4": (P.density_cube(20000, 16.0, seed=3), 0.0),
        "dense_K8": (P.density_cube(20000, 40.0, seed=4), 0.0),
        "margin": (P.jittered_lattice(9999, 22, 9.0, 1.5, 9.0, 11.0, 5), 1.5),
        "faces": (face, 0.0),
        "slab": (slab, 0.0),
        "near_origin": (near, 0.0),
    }


@pytest.mark.parametrize("name", list(_cases()))
def test_windowed_walk_is_bit_identical_to_full_runs(U, name):
    st, margin = _cases()[name]
    prm = U.Params(contact_margin=margin)
    _same(U, st, prm)


@pytest.mark.parametrize("nbar", [8, 64])
def test_windowed_walk_full_size(U, nbar):
    """4,194,304 cells at a mean of 8 and 64 overlapping neighbours (2 and 8
    slices per box), two fused steps, as the density sweep runs them."""
    st = P.density_cube(1 << 22, float(nbar), seed=nbar)
    _same(U, st, U.Params(max_disp=0.0), nsteps=2, ways=("step", "batched_full_runs",
                                                          "batched_windows"))


def test_per_box_entry_points_ignore_reserved(U):
    """ug_compute_forces reads a caller's per-box table; a geometry record whose
    reserved word is not 0 must not change how it is read."""
    st = P.density_cube(8000, 16.0, seed=9)
    x = torch.from_numpy(st).to(DEV)
    srt, perm, start, info, _ = U.grid_build(x)
    assert U.grid_info_from_bytes(info)["reserved"] == 0
    F = U.compute_forces(srt, start, info, U.Params())
    info2 = info.clone()
    info2[44:48] = torch.tensor([3, 0, 0, 0], dtype=torch.uint8, device=DEV)
    F2 = U.compute_forces(srt, start, info2, U.Params())
    assert torch.equal(F, F2)


def _run_pairs_once(U, st, prm, nsteps, walk, offs=None):
    x = torch.from_numpy(np.ascontiguousarray(st, np.float32)).to(DEV)
    n = x.shape[0]
    if offs is None:
        offs = np.array([0, n])
    nsims = len(offs) - 1
    parts = [x[int(offs[k]):int(offs[k + 1])] for k in range(nsims)]
    mb = sum(U.estimate_max_boxes(p, prm.contact_margin, slack=2.0, extra_extent=8.0 * nsteps)
             for p in parts)
    sp = U.Stepper(n, mb, x.device, nsims=nsims)
    perm = U.iota(n, x.device)
    if walk == "step":
        sp.step(x, perm, prm, nsteps, pairs_once=True)
    else:
        t = U.ug_tuning()
        t.agents_per_lane, t.sweep_block, t.pair_mode = 2, 128, 1
        t.neighbour_walk = {"full_runs": 1, "windows": 2, "default": 0}[walk]
        o = torch.from_numpy(np.asarray(offs, np.int32)).to(DEV)
        sp.step_batched(x, perm, o, torch.stack([prm.as_tensor(DEV)] * nsims), nsteps, t)
    sp.check()
    return x, perm


@pytest.mark.parametrize("name", list(_cases()))
def test_pairs_once_windows_are_bit_identical_to_full_runs(U, name):
    st, margin = _cases()[name]
    prm = U.Params(contact_margin=margin)
    a, pa = _run_pairs_once(U, st, prm, 3, "step")
    for how in ("full_runs", "windows", "default"):
        b, pb = _run_pairs_once(U, st, prm, 3, how)
        assert torch.equal(pa, pb), how
        assert torch.equal(a, b), how


def test_pairs_once_windows_several_simulations(U):
    """Three simulations of 1, 2 and 8 x slices per box in one batched call:
    windows and full runs give the same bits."""
    sts = [P.density_cube(6000, 2.0, seed=11), P.density_cube(9000, 16.0, seed=12),
           P.density_cube(7001, 40.0, seed=13)]
    st = np.concatenate(sts)
    offs = np.cumsum([0] + [len(t) for t in sts])
    prm = U.Params()
    a, pa = _run_pairs_once(U, st, prm, 3, "full_runs", offs)
    b, pb = _run_pairs_once(U, st, prm, 3, "windows", offs)
    assert torch.equal(pa, pb)
    assert torch.equal(a, b)


def test_pairs_once_windows_full_size(U):
    """4,194,304 cells at a mean of 64 overlapping neighbours, two steps."""
    st = P.density_cube(1 << 22, 64.0, seed=64)
    prm = U.Params(max_disp=0.0)
    a, pa = _run_pairs_once(U, st, prm, 2, "full_runs")
    b, pb = _run_pairs_once(U, st, prm, 2, "windows")
    assert torch.equal(pa, pb)
    assert torch.equal(a, b)
