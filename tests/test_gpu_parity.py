"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Exact: grid geometry, box table, the stable box order (permutation), contact
pair sets.  Within TOL_STEP = 1e-5 (condition-scaled, see _metrics): forces and
displacements per step.  Within TOL_TRAJ = 1e-3: positions after 100 steps.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2105_00039_gb300 import populations as P

from _metrics import (TOL_STEP, TOL_TRAJ, adherence_flips, by_id, disp_errors, force_errors,
                      ulp32)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def U():
    from paper_2105_00039_gb300 import ugmech
    ugmech.load()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return ugmech


DEV = "cuda"


def workloads():
    return {
        "uniform4096": (P.small_uniform(0), 0.0),
        "lattice4096_margin": (P.jittered_lattice(4096, 16, 9.0, 1.5, 9.0, 11.0, 1), 1.5),
        "dense_cube": (P.uniform_cube(3000, 60.0, 8.0, 12.0, 2), 0.0),
        "ragged_777": (P.uniform_cube(777, 70.0, 8.0, 12.0, 3), 0.0),
    }


def _gpu(st):
    return torch.from_numpy(np.ascontiguousarray(st, np.float32)).to(DEV)


# ------------------------------------------------------------------ grid
@pytest.mark.parametrize("name", list(workloads()))
def test_grid_build_exact(U, name):
    st, margin = workloads()[name]
    g = O.grid(st, margin)
    srt, perm, start, info, _ = U.grid_build(_gpu(st), contact_margin=margin,
                                             max_boxes=g["nboxes"] + 5)
    gi = U.grid_info_from_bytes(info)
    assert np.array_equal(np.float32(gi["origin"]), g["origin"])
    assert np.float32(gi["edge"]) == g["edge"]
    assert gi["dims"] == list(g["dims"]) and gi["nboxes"] == g["nboxes"]
    assert np.array_equal(start.cpu().numpy()[: g["nboxes"] + 1], g["start"])
    assert np.array_equal(perm.cpu().numpy(), g["perm"])
    assert np.array_equal(srt.cpu().numpy(), st[g["perm"]])


def test_grid_build_with_input_ids(U):
    st = P.small_uniform(4)
    ids = np.random.default_rng(0).permutation(len(st)).astype(np.int32)
    g = O.grid(st)
    _, perm, _, _, _ = U.grid_build(_gpu(st), torch.from_numpy(ids).to(DEV))
    assert np.array_equal(perm.cpu().numpy(), ids[g["perm"]])


def test_grid_build_exact_many_scan_tiles(U):
    """2^21 agents on 140^3 = 2.7M boxes: 335 scan tiles of 8192 boxes, each
    taking its prefix from the earlier tiles' row counts."""
    st = P.density_cube(1 << 21, 2.0, seed=21)
    g = O.grid(st)
    assert g["nboxes"] > 300 * 8192
    srt, perm, start, info, _ = U.grid_build(_gpu(st), max_boxes=g["nboxes"] + 7)
    assert U.grid_info_from_bytes(info)["nboxes"] == g["nboxes"]
    assert np.array_equal(start.cpu().numpy()[: g["nboxes"] + 1], g["start"])
    assert np.array_equal(perm.cpu().numpy(), g["perm"])
    assert np.array_equal(srt.cpu().numpy(), st[g["perm"]])


# ------------------------------------------------------------------ pairs
@pytest.mark.parametrize("name", list(workloads()))
def test_contact_pairs_exact(U, name):
    st, margin = workloads()[name]
    srt, perm, start, info, _ = U.grid_build(_gpu(st), contact_margin=margin)
    count, nbr = U.list_pairs(srt, start, info, margin, max_per_agent=256)
    pid = perm.cpu().numpy()
    c = count.cpu().numpy()
    nb = nbr.cpu().numpy()
    gpu = set()
    for s in range(len(st)):
        for j in nb[s, : c[s]]:
            gpu.add((int(pid[s]), int(pid[j])))
    pos, rad = st[:, :3].astype(np.float64), 0.5 * st[:, 3].astype(np.float64)
    I, J = O.pairs_bruteforce(pos, rad, margin)
    ref = set(zip(I.tolist(), J.tolist()))
    # pairs within 1e-9 of contact may go either way (none expected)
    d = np.linalg.norm(pos[I] - pos[J], axis=1)
    assert gpu == ref, (len(gpu - ref), len(ref - gpu))
    assert len(ref) > 0


def test_list_capacity_error(U):
    st = P.uniform_cube(500, 25.0, 8.0, 12.0, 5)        # very dense: many contacts each
    srt, perm, start, info, status = U.grid_build(_gpu(st))
    with pytest.raises(U.UgError) as e:
        U.list_pairs(srt, start, info, 0.0, max_per_agent=4)
    assert e.value.code == U.UG_ECAPACITY


# ------------------------------------------------------------------ forces / displacement
@pytest.mark.parametrize("name", list(workloads()))
def test_forces_parity(U, name):
    st, margin = workloads()[name]
    prm = O.Params(contact_margin=margin)
    srt, perm, start, info, _ = U.grid_build(_gpu(st), contact_margin=margin)
    F = U.compute_forces(srt, start, info, U.Params(contact_margin=margin))
    pid = perm.cpu().numpy()
    Fg = by_id(F.cpu().numpy().astype(np.float64), pid)
    ref = O.step(st, prm)
    per, norm, bad_zero = force_errors(Fg[:, :3], ref["F"], ref["S"])
    assert per <= TOL_STEP and norm <= TOL_STEP and bad_zero == 0, (per, norm, bad_zero)
    assert np.array_equal(Fg[:, 3].astype(np.int64), ref["npairs"])


@pytest.mark.parametrize("name", list(workloads()))
def test_displacement_parity(U, name):
    st, margin = workloads()[name]
    prm = O.Params(contact_margin=margin, max_disp=0.5)
    uprm = U.Params(contact_margin=margin, max_disp=0.5)
    srt, perm, start, info, _ = U.grid_build(_gpu(st), contact_margin=margin)
    F = U.compute_forces(srt, start, info, uprm)
    new, disp = U.apply_displacement(srt, F, uprm)
    pid = perm.cpu().numpy()
    ug = by_id(disp.cpu().numpy().astype(np.float64), pid)
    newg = by_id(new.cpu().numpy().astype(np.float64), pid)
    ref = O.step(st, prm)
    flips = adherence_flips(ref["Fn"], ref["S"], prm.adherence)
    assert flips.sum() <= 1
    per, bad_zero = disp_errors(ug[:, :3], ref["u"], ref["S"], st[:, 3], exclude=flips)
    assert per <= TOL_STEP and bad_zero == 0, (per, bad_zero)
    assert np.array_equal(ug[~flips, 3] > 0, ref["moving"][~flips])
    assert ref["capped"].any()
    # new position = float32(p + u): within one ulp of p + u_ref plus the u error
    scale = np.linalg.norm(ref["u"], axis=1)[:, None] + 1e-30
    dp = np.abs(newg[:, :3] - (st[:, :3].astype(np.float64) + ref["u"]))
    ok = dp <= ulp32(newg[:, :3]) + 2 * TOL_STEP * np.maximum(scale, 1e-3)
    assert ok[~flips].all()
    assert np.array_equal(newg[:, 3], st[:, 3].astype(np.float64))


# ------------------------------------------------------------------ fused step
def _run_steps(U, st, prm, nsteps, max_boxes=None, pairs_once=False):
    x = _gpu(st)
    n = len(st)
    if max_boxes is None:
        max_boxes = U.estimate_max_boxes(x, prm.contact_margin, slack=2.0)
    sp = U.Stepper(n, max_boxes, x.device)
    perm = U.iota(n, x.device)
    sp.step(x, perm, prm, nsteps, pairs_once=pairs_once)
    sp.check()
    return x.cpu().numpy(), perm.cpu().numpy()


@pytest.mark.parametrize("pairs_once", [False, True])
@pytest.mark.parametrize("name", list(workloads()))
def test_fused_single_step(U, name, pairs_once):
    st, margin = workloads()[name]
    prm = O.Params(contact_margin=margin)
    out, perm = _run_steps(U, st, U.Params(contact_margin=margin), 1, pairs_once=pairs_once)
    g = O.grid(st, margin)
    assert np.array_equal(perm, g["perm"])          # rows come back in the step's box order
    newg = by_id(out.astype(np.float64), perm)
    ref = O.step(st, prm)
    flips = adherence_flips(ref["Fn"], ref["S"], prm.adherence)
    scale = ref["S"] / O.mass(st[:, 3].astype(np.float64), prm.as64())
    dp = np.abs(newg[:, :3] - ref["state"][:, :3])
    ok = dp <= ulp32(newg[:, :3]) + TOL_STEP * np.maximum(np.linalg.norm(ref["u"], axis=1),
                                                          scale)[:, None]
    assert ok[~flips].all(), np.argwhere(~ok)[:5]


@pytest.mark.parametrize("pairs_once", [False, True])
def test_fused_step_is_deterministic(U, pairs_once):
    st = P.uniform_cube(20000, 250.0, 8.0, 12.0, 9)
    a, pa = _run_steps(U, st, U.Params(), 5, pairs_once=pairs_once)
    b, pb = _run_steps(U, st, U.Params(), 5, pairs_once=pairs_once)
    assert np.array_equal(a, b) and np.array_equal(pa, pb)


@pytest.mark.parametrize("pairs_once", [False, True])
def test_trajectory_100_steps(U, pairs_once):
    """100 independent steps on both sides, no adherence threshold (the step is
    then continuous in the rows, so float32 and FP64 trajectories stay close)."""
    st = P.lattice_cube(16, seed=0)                    # 4096 cells, same recipe as the 1M lattice
    prm = O.Params(adherence=0.0)
    out, perm = _run_steps(U, st, U.Params(adherence=0.0), 100, pairs_once=pairs_once)
    final_g = by_id(out.astype(np.float64), perm)[:, :3]
    final_r, recs = O.trajectory(st, prm, 100, keep=True)
    mean_u = np.mean([np.linalg.norm(r["u"], axis=1).mean() for r in recs])
    err = np.linalg.norm(final_g - final_r[:, :3], axis=1) / (mean_u * 100)
    assert err.max() <= TOL_TRAJ, (err.max(), mean_u)


def _stepwise_states(U, st, prm_u, nsteps):
    """The GPU's rows (by id) before every step, one ug_step call per step."""
    x = _gpu(st)
    n = len(st)
    mb = U.estimate_max_boxes(x, prm_u.contact_margin, slack=3.0)
    sp = U.Stepper(n, mb, x.device)
    perm = U.iota(n, x.device)
    states = [st.copy()]
    for _ in range(nsteps):
        sp.step(x, perm, prm_u, 1)
        states.append(U.scatter_rows(x, perm).cpu().numpy())
    sp.check()
    return states, mb


def test_trajectory_100_steps_shadowed(U):
    """With the default adherence threshold, every one of 100 steps is checked
    against the oracle applied to the GPU's own input rows (the per-step
    tolerance, adherence-threshold ties excluded), and the fused 100-step call
    reproduces the step-by-step rows bit for bit."""
    st = P.lattice_cube(16, seed=0)
    prm = O.Params()
    states, mb = _stepwise_states(U, st, U.Params(), 100)
    flips_total = 0
    for t in range(100):
        X, Y = states[t], states[t + 1]
        ref = O.step(X, prm)
        flips = adherence_flips(ref["Fn"], ref["S"], prm.adherence)
        flips_total += int(flips.sum())
        scale = ref["S"] / O.mass(X[:, 3].astype(np.float64), prm.as64())
        dp = np.abs(Y[:, :3].astype(np.float64) - ref["state"][:, :3])
        ok = dp <= ulp32(Y[:, :3]) + TOL_STEP * np.maximum(np.linalg.norm(ref["u"], axis=1),
                                                            scale)[:, None]
        assert ok[~flips].all(), (t, np.argwhere(~ok)[:5])
        # an agent whose |F| ties with the threshold either stayed put or moved
        # by the oracle's (capped) v; both are correct decisions within rounding
        stayed = np.all(Y[flips, :3] == X[flips, :3], axis=1)
        v, vn = ref["v"][flips], ref["vn"][flips]
        u_move = v * np.minimum(1.0, prm.as64().max_disp / np.maximum(vn, 1e-300))[:, None]
        dm = np.abs(Y[flips, :3].astype(np.float64) - (X[flips, :3].astype(np.float64) + u_move))
        moved = np.all(dm <= ulp32(Y[flips, :3]) + TOL_STEP * np.maximum(
            np.linalg.norm(u_move, axis=1), scale[flips])[:, None], axis=1)
        assert (stayed | moved).all(), t
    assert flips_total <= 0.02 * 100 * len(st)
    out, perm = _run_steps(U, st, U.Params(), 100, max_boxes=mb)
    assert np.array_equal(by_id(out, perm), states[-1])


def test_freeze_rule_max_disp_zero(U):
    st = P.density_cube(50000, 8.0, seed=4)
    out, perm = _run_steps(U, st, U.Params(max_disp=0.0), 20)
    assert np.array_equal(by_id(out, perm), st)


# ------------------------------------------------------------------ batched
@pytest.mark.parametrize("pairs_once", [False, True])
def test_batched_bit_identical_to_plain(U, pairs_once):
    rng_sizes = [1500, 37, 8000, 2600, 1, 12000, 640, 5000]
    parts = [P.density_cube(n, 4.0 + 6.0 * k, seed=100 + k) for k, n in enumerate(rng_sizes)]
    offs = np.zeros(len(parts) + 1, np.int64)
    offs[1:] = np.cumsum([len(p) for p in parts])
    st = np.concatenate(parts)
    params = [U.Params(k=2.0 + 0.1 * k, gamma=1.0, contact_margin=0.25 * (k % 3)) for k in range(len(parts))]
    x = _gpu(st)
    n = len(st)
    per_sim_boxes = [U.estimate_max_boxes(_gpu(p), params[k].contact_margin, slack=2.0)
                     for k, p in enumerate(parts)]
    mb = sum(per_sim_boxes)
    sp = U.Stepper(n, mb, x.device, nsims=len(parts))
    perm = U.iota(n, x.device)
    off_t = torch.from_numpy(offs.astype(np.int32)).to(DEV)
    pdev = torch.stack([p.as_tensor(DEV) for p in params])
    t = U.ug_tuning()
    t.pair_mode = 1 if pairs_once else 0
    sp.step_batched(x, perm, off_t, pdev, nsteps=7, tuning=t)
    sp.check("batched")
    xb, pb = x.cpu().numpy(), perm.cpu().numpy()
    for k, part in enumerate(parts):
        a, b = offs[k], offs[k + 1]
        out, pp = _run_steps(U, part, params[k], 7, max_boxes=per_sim_boxes[k], pairs_once=pairs_once)
        assert np.array_equal(xb[a:b], out), k
        assert np.array_equal(pb[a:b] - a, pp), k


def test_batched_empty_simulations(U):
    parts = [P.density_cube(3000, 8.0, seed=7), np.zeros((0, 4), np.float32),
             P.density_cube(2000, 16.0, seed=8), np.zeros((0, 4), np.float32)]
    offs = np.zeros(len(parts) + 1, np.int64)
    offs[1:] = np.cumsum([len(p) for p in parts])
    st = np.concatenate(parts)
    x = _gpu(st)
    sp = U.Stepper(len(st), 200000, x.device, nsims=len(parts))
    perm = U.iota(len(st), x.device)
    pdev = torch.stack([U.Params().as_tensor(DEV) for _ in parts])
    sp.step_batched(x, perm, torch.from_numpy(offs.astype(np.int32)).to(DEV), pdev, nsteps=2)
    sp.check("batched-empty")
    for k in (0, 2):
        out, pp = _run_steps(U, parts[k], U.Params(), 2, max_boxes=100000)
        assert np.array_equal(x.cpu().numpy()[offs[k]:offs[k + 1]], out)


def test_autotuner_picks_a_valid_block(U):
    st, offs = P.batched_population(nsims=6, nmin=1000, nmax=20000, seed=3)
    x = _gpu(st)
    pdev = torch.stack([U.Params().as_tensor(DEV) for _ in range(6)])
    best = U.tune_batched(x, torch.from_numpy(offs.astype(np.int32)).to(DEV), pdev, 6, 2_000_000)
    assert (best.agents_per_lane, best.sweep_block) in ((1, 64), (1, 128), (2, 128))
    assert best.pair_mode in (0, 1)
    # every configuration gives the same bits
    outs = []
    for apl, blk in ((1, 64), (1, 128), (2, 128)):
        t = U.ug_tuning()
        t.agents_per_lane, t.sweep_block = apl, blk
        y = x.clone()
        perm = U.iota(len(st), x.device)
        sp = U.Stepper(len(st), 2_000_000, x.device, nsims=6)
        sp.step_batched(y, perm, torch.from_numpy(offs.astype(np.int32)).to(DEV), pdev, 3, t)
        sp.check("tuned")
        outs.append(y.cpu().numpy())
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


# ------------------------------------------------------------------ edge cases
def test_single_agent_and_pair(U):
    one = np.array([[5.0, -3.0, 2.0, 10.0]], np.float32)
    out, perm = _run_steps(U, one, U.Params(), 3)
    assert np.array_equal(out, one)
    two = np.array([[0, 0, 0, 10], [9, 0, 0, 10]], np.float32)
    srt, perm, start, info, _ = U.grid_build(_gpu(two))
    F = by_id(U.compute_forces(srt, start, info).cpu().numpy(), perm.cpu().numpy())
    np.testing.assert_allclose(F[:, 0], [-0.41886116991581024, 0.41886116991581024], rtol=2e-6)


def test_coincident_centres_contribute_nothing(U):
    st = np.array([[1, 2, 3, 10], [1, 2, 3, 10], [8, 2, 3, 10]], np.float32)
    srt, perm, start, info, _ = U.grid_build(_gpu(st))
    F = by_id(U.compute_forces(srt, start, info).cpu().numpy().astype(np.float64), perm.cpu().numpy())
    ref = O.step(st, O.Params(), method="brute")
    np.testing.assert_allclose(F[:, :3], ref["F"], rtol=1e-6, atol=1e-7)
    assert list(F[:, 3]) == [1, 1, 2]


def test_everything_in_one_box(U):
    st = P.uniform_cube(400, 4.0, 10.0, 10.0, 11)         # 400 agents in a 4^3 cube
    ref = O.step(st, O.Params())
    srt, perm, start, info, _ = U.grid_build(_gpu(st))
    F = by_id(U.compute_forces(srt, start, info).cpu().numpy().astype(np.float64), perm.cpu().numpy())
    per, norm, bad = force_errors(F[:, :3], ref["F"], ref["S"])
    assert per <= TOL_STEP and bad == 0
    assert np.all(F[:, 3] == 399)


def test_agents_on_box_faces(U):
    # centres exactly on multiples of the box edge (edge 8, origin -8 after rounding)
    g = np.stack(np.meshgrid(*[np.arange(0, 64, 8.0)] * 3, indexing="ij"), -1).reshape(-1, 3)
    st = np.concatenate([g, np.full((len(g), 1), 8.0)], axis=1).astype(np.float32)
    st[::7, 3] = 7.5
    ref_g = O.grid(st)
    srt, perm, start, info, _ = U.grid_build(_gpu(st))
    assert np.array_equal(perm.cpu().numpy(), ref_g["perm"])
    F = by_id(U.compute_forces(srt, start, info).cpu().numpy().astype(np.float64), perm.cpu().numpy())
    ref = O.step(st, O.Params())
    assert np.array_equal(F[:, 3].astype(int), ref["npairs"])


def test_negative_and_large_coordinates(U):
    st = P.uniform_cube(3000, 200.0, 8.0, 12.0, 12)
    st[:, :3] -= np.float32(1.0e4)
    ref = O.step(st, O.Params())
    srt, perm, start, info, _ = U.grid_build(_gpu(st))
    F = by_id(U.compute_forces(srt, start, info).cpu().numpy().astype(np.float64), perm.cpu().numpy())
    per, norm, bad = force_errors(F[:, :3], ref["F"], ref["S"])
    assert per <= TOL_STEP and bad == 0, per


def test_grid_too_large_is_reported(U):
    st = P.uniform_cube(100, 50.0, 8.0, 12.0, 13)
    st[0, :3] = 1.0e5
    with pytest.raises(U.UgError) as e:
        U.grid_build(_gpu(st), max_boxes=100000)
    assert e.value.code == U.UG_EGRID_TOO_LARGE
    x = _gpu(st)
    sp = U.Stepper(100, 100000, x.device)
    perm = U.iota(100, x.device)
    sp.step(x, perm, U.Params(), 3)
    with pytest.raises(U.UgError) as e:
        sp.check()
    assert e.value.code == U.UG_EGRID_TOO_LARGE


@pytest.mark.parametrize("bad", ["nan", "inf", "zero_diameter", "negative_diameter"])
def test_bad_state_is_reported(U, bad):
    st = P.uniform_cube(300, 50.0, 8.0, 12.0, 14)
    if bad == "nan":
        st[17, 1] = np.nan
    elif bad == "inf":
        st[17, 2] = np.inf
    elif bad == "zero_diameter":
        st[17, 3] = 0.0
    else:
        st[17, 3] = -1.0
    with pytest.raises(U.UgError) as e:
        U.grid_build(_gpu(st), max_boxes=100000)
    assert e.value.code == U.UG_EBADSTATE


def test_simulate_host_round_trip(U):
    st = P.small_uniform(2)
    out = U.simulate(torch.from_numpy(st), U.Params(), nsteps=1)
    assert out.device.type == "cpu"
    ref = O.step(st, O.Params())
    flips = adherence_flips(ref["Fn"], ref["S"], 0.1)
    dp = np.abs(out.numpy()[:, :3].astype(np.float64) - ref["state"][:, :3])
    assert (dp[~flips] <= ulp32(out.numpy()[~flips, :3]) + 1e-5).all()


# ------------------------------------------------------------------ full-size, sampled
def _sampled_check(U, x, prm_o, prm_u, nsample=3000, seed=0, symmetric=False):
    """Grid + forces of the GPU's own current rows, compared agent by agent
    with the oracle on a random sample of agents; with symmetric=True the
    every-pair-once forces (ug_forces_symmetric) of the same grid as well."""
    srt, perm, start, info, _ = U.grid_build(x, contact_margin=prm_u.contact_margin,
                                             max_boxes=U.estimate_max_boxes(x, prm_u.contact_margin))
    forces = [U.compute_forces(srt, start, info, prm_u)]
    if symmetric:
        forces.append(U.forces_symmetric(srt, start, info, prm_u))
    st = x.cpu().numpy()
    pid = perm.cpu().numpy()
    idx = np.random.default_rng(seed).choice(len(st), size=min(nsample, len(st)), replace=False)
    ref = O.step_sampled(st, idx, prm_o)
    for F in forces:
        Fg = by_id(F.cpu().numpy().astype(np.float64), pid)
        per, norm, bad = force_errors(Fg[idx, :3], ref["F"], ref["S"])
        assert per <= TOL_STEP and bad == 0, (per, bad)
        assert np.array_equal(Fg[idx, 3].astype(np.int64), ref["npairs"])
        tot = Fg[:, :3].sum(0)
        assert np.abs(tot).max() <= 1e-4 * np.abs(Fg[:, :3]).sum(0).max()   # Newton's third law
    return float(ref["npairs"].mean())


@pytest.mark.parametrize("pairs_once", [False, True])
def test_full_size_lattice_1m_100_steps(U, pairs_once):
    """The benchmark's configuration: 2^20 lattice cells, 100 fused steps (the
    gather step or every pair once); the rows the GPU holds before the first
    and after the last step are checked agent by agent."""
    st = P.lattice_1m(0)
    x = _gpu(st)
    n = len(st)
    mb = U.estimate_max_boxes(x, 0.0, slack=1.5)
    nb0 = _sampled_check(U, x, O.Params(), U.Params())
    assert 3.0 < nb0 < 7.0
    sp = U.Stepper(n, mb, x.device)
    perm = U.iota(n, x.device)
    sp.step(x, perm, U.Params(), 100, pairs_once=pairs_once)
    sp.check()
    p = perm.cpu().numpy()
    assert np.array_equal(np.sort(p), np.arange(n))
    _sampled_check(U, x, O.Params(), U.Params(), seed=1)


@pytest.mark.parametrize("n,nbar", [(1 << 22, 2), (1 << 22, 8), (1 << 22, 32), (1 << 22, 64),
                                    (1 << 24, 12)])
def test_density_sweep_sampled(U, n, nbar):
    """The density sweep's populations at full size (4M cells at 2 to 64 mean
    neighbours, 16M at 12, the seeds the benchmark uses): gather and
    every-pair-once forces against the oracle on a sample of agents."""
    st = P.density_cube(n, float(nbar), seed=nbar)
    x = _gpu(st)
    nb = _sampled_check(U, x, O.Params(max_disp=0.0), U.Params(max_disp=0.0), nsample=1500,
                        symmetric=True)
    assert 0.6 * nbar < nb < 1.2 * nbar


@pytest.mark.parametrize("pairs_once", [False, True])
def test_batched_full_population(U, pairs_once):
    """The batched workload at full size: 256 simulations (log-uniform counts in
    [1e3, 2e5], mean neighbours U[4, 40]).  One batched step against the oracle
    on a sample of agents of four simulations, then 50 batched steps bit for bit
    against each simulation run alone with the plain step of the same method."""
    nsims = 256
    st, offs = P.batched_population(nsims=nsims, seed=0)
    n = len(st)
    x0 = _gpu(st)
    offs_t = torch.from_numpy(offs.astype(np.int32)).to(DEV)
    prm = U.Params()
    pdev = torch.stack([prm.as_tensor(DEV) for _ in range(nsims)])
    caps = [4 * U.estimate_max_boxes(x0[int(offs[k]):int(offs[k + 1])], 0.0, slack=1.0,
                                     extra_extent=24.0) + 1000 for k in range(nsims)]
    sp = U.Stepper(n, int(sum(caps)), x0.device, nsims=nsims)
    t = U.ug_tuning()
    t.pair_mode = 1 if pairs_once else 0
    # one step against the oracle
    x = x0.clone()
    perm = U.iota(n, x.device)
    sp.step_batched(x, perm, offs_t, pdev, 1, t)
    sp.check("batched-1")
    new = by_id(x.cpu().numpy().astype(np.float64), perm.cpu().numpy())
    rng = np.random.default_rng(1)
    for k in (0, 85, 170, 255):
        a, b = int(offs[k]), int(offs[k + 1])
        part = st[a:b]
        idx = rng.choice(b - a, size=min(300, b - a), replace=False)
        ref = O.step_sampled(part, idx, O.Params())
        flips = adherence_flips(ref["Fn"], ref["S"], 0.1)
        scale = ref["S"] / O.mass(part[idx, 3].astype(np.float64), O.Params().as64())
        got = new[a:b][idx, :3]
        want = part[idx, :3].astype(np.float64) + ref["u"]
        ok = np.abs(got - want) <= ulp32(got) + TOL_STEP * np.maximum(
            np.linalg.norm(ref["u"], axis=1), scale)[:, None]
        assert ok[~flips].all(), (k, np.argwhere(~ok)[:5])
    # 50 steps, batched vs alone
    x = x0.clone()
    perm = U.iota(n, x.device)
    sp.step_batched(x, perm, offs_t, pdev, 50, t)
    sp.check("batched-50")
    xb, pb = x.cpu().numpy(), perm.cpu().numpy()
    for k in range(nsims):
        a, b = int(offs[k]), int(offs[k + 1])
        y = x0[a:b].clone()
        py = U.iota(b - a, y.device)
        alone = U.Stepper(b - a, caps[k], y.device)
        alone.step(y, py, prm, 50, pairs_once=pairs_once)
        alone.check("alone")
        assert np.array_equal(xb[a:b], y.cpu().numpy()), k
        assert np.array_equal(pb[a:b] - a, py.cpu().numpy()), k


def _thin_slab(n, thickness, side, seed):
    """Uniform centres in [0, thickness] x [0, side]^2, diameters U[8, 12]:
    a grid only 3 or 4 boxes wide in x, where most pairs of consecutive agents
    must not share a merged run."""
    st = P.uniform_cube(n, side, 8.0, 12.0, seed)
    st[:, 0] = st[:, 0] * np.float32(thickness / side)
    return st


@pytest.mark.parametrize("name", ["dense", "slab_x3", "slab_x4"])
def test_step_against_oracle_and_one_agent_kernel(U, name):
    """Dense grids (about 24 agents per box, ~60 neighbours) and grids 3 or 4
    boxes wide in x: one fused step against the oracle, and three steps bit for
    bit against the one-agent-per-lane sweep of the batched entry."""
    st = {"dense": lambda: P.density_cube(20000, 60.0, seed=31),
          "slab_x3": lambda: _thin_slab(6000, 5.0, 600.0, 32),
          "slab_x4": lambda: _thin_slab(6000, 14.0, 600.0, 33)}[name]()
    if name != "dense":
        g = O.grid(st)
        assert g["dims"][0] == (3 if name == "slab_x3" else 4)
    prm = O.Params()
    out, perm = _run_steps(U, st, U.Params(), 1)
    newg = by_id(out.astype(np.float64), perm)
    ref = O.step(st, prm)
    flips = adherence_flips(ref["Fn"], ref["S"], prm.adherence)
    scale = ref["S"] / O.mass(st[:, 3].astype(np.float64), prm.as64())
    dp = np.abs(newg[:, :3] - ref["state"][:, :3])
    ok = dp <= ulp32(newg[:, :3]) + TOL_STEP * np.maximum(np.linalg.norm(ref["u"], axis=1),
                                                          scale)[:, None]
    assert ok[~flips].all()
    assert ref["npairs"].mean() > 2.0
    # three steps: two agents per lane (plain) == one agent per lane (batched, 1 simulation)
    a, pa = _run_steps(U, st, U.Params(), 3)
    x = _gpu(st)
    t = U.ug_tuning()
    t.agents_per_lane, t.sweep_block = 1, 128
    sp = U.Stepper(len(st), U.estimate_max_boxes(x, 0.0, slack=2.0), x.device, nsims=1)
    pb = U.iota(len(st), x.device)
    sp.step_batched(x, pb, torch.tensor([0, len(st)], dtype=torch.int32, device=DEV),
                    U.Params().as_tensor(DEV)[None], 3, t)
    sp.check("batched-1")
    assert np.array_equal(a, x.cpu().numpy()) and np.array_equal(pa, pb.cpu().numpy())


@pytest.mark.parametrize("name", ["dense", "slab_x3", "slab_x4"])
def test_pairs_once_step_against_oracle(U, name):
    """ug_step_pairs_once on a dense grid and on grids 3 or 4 boxes wide in x:
    one step against the oracle, and three steps against the gather step
    within the per-step tolerance of the displacements."""
    st = {"dense": lambda: P.density_cube(20000, 60.0, seed=31),
          "slab_x3": lambda: _thin_slab(6000, 5.0, 600.0, 32),
          "slab_x4": lambda: _thin_slab(6000, 14.0, 600.0, 33)}[name]()
    prm = O.Params()
    out, perm = _run_steps(U, st, U.Params(), 1, pairs_once=True)
    newg = by_id(out.astype(np.float64), perm)
    ref = O.step(st, prm)
    flips = adherence_flips(ref["Fn"], ref["S"], prm.adherence)
    scale = ref["S"] / O.mass(st[:, 3].astype(np.float64), prm.as64())
    dp = np.abs(newg[:, :3] - ref["state"][:, :3])
    ok = dp <= ulp32(newg[:, :3]) + TOL_STEP * np.maximum(np.linalg.norm(ref["u"], axis=1),
                                                          scale)[:, None]
    assert ok[~flips].all()
    a, pa = _run_steps(U, st, U.Params(adherence=0.0), 3, pairs_once=True)
    b, pb = _run_steps(U, st, U.Params(adherence=0.0), 3)
    ga, gb = by_id(a.astype(np.float64), pa), by_id(b.astype(np.float64), pb)
    assert np.abs(ga[:, :3] - gb[:, :3]).max() < 1e-3


@pytest.mark.parametrize("pairs_once", [False, True])
def test_stepper_room_serves_smaller_populations(U, pairs_once):
    """A Stepper sized for n agents steps any population of up to n (agents
    added or removed between calls), with the same bits as one sized exactly,
    and refuses a larger one before any device work."""
    st = P.small_uniform(4)
    big = U.Stepper(len(st), 200000, torch.device(DEV))
    for m in (3000, 4096, 1234):
        part = st[:m]
        x = _gpu(part)
        perm = U.iota(m, x.device)
        big.step(x, perm, U.Params(), 3, pairs_once=pairs_once)
        big.check()
        ref, pref = _run_steps(U, part, U.Params(), 3, max_boxes=200000, pairs_once=pairs_once)
        assert np.array_equal(x.cpu().numpy(), ref) and np.array_equal(perm.cpu().numpy(), pref)
    small = U.Stepper(100, 200000, torch.device(DEV))
    x = _gpu(st[:101])
    with pytest.raises(ValueError):
        small.step(x, U.iota(101, x.device), U.Params(), 1)
    with pytest.raises(ValueError):
        small.step(_gpu(st[:50]), U.iota(60, x.device), U.Params(), 1)


@pytest.mark.parametrize("pairs_once", [False, True])
def test_simulation_run_host_to_host(U, pairs_once):
    """The end-to-end API: host rows in id order in, host rows in id order out,
    the same bits as the device-side steps."""
    st = P.small_uniform(6)
    n = len(st)
    mb = U.estimate_max_boxes(_gpu(st), 0.0, slack=2.0)
    sim = U.Simulation(n, mb, DEV)
    host_in = torch.from_numpy(st).pin_memory()
    out = sim.run(host_in, U.Params(), 4, pairs_once=pairs_once).numpy().copy()
    dev, perm = _run_steps(U, st, U.Params(), 4, max_boxes=mb, pairs_once=pairs_once)
    assert np.array_equal(out, by_id(dev, perm))
    again = sim.run(host_in, U.Params(), 4, pairs_once=pairs_once).numpy()
    assert np.array_equal(out, again)                 # buffers reused, same result
