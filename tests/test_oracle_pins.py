"""Pins for the FP64 oracle: it is checked against things other than itself.

  * worked examples of Eq. 1 derived by hand (tests/golden/eq1_worked_examples.json);
  * the force as minus the gradient of the pair potential
    V(delta) = kappa delta^2/2 - (2/3) gamma sqrt(R) delta^(3/2), whose derivative
    in delta is Eq. 1's magnitude (an independent route to the same numbers);
  * Newton's third law, rotation/permutation/scaling invariance;
  * brute-force pair search as the definition of the kd-tree search;
  * closed-form displacements (Sec. III rules as read here: strict adherence,
    u = (dt / m) F with m = density (pi/6) d^3, the cap along u), with dt != 1
    and a capped case;
  * a hand-worked grid (edge, padding layer, x-fastest keys, exclusive starts),
    the x slices that order agents inside a box (the density rule's
    thresholds, a hand-worked order) and the slice order on random populations
    and the uniform grid's completeness condition (Sec. IV-A): every contact
    pair lies in adjacent boxes;
  * the adjoint against FP64 central finite differences of the forward, on
    fixtures with capped agents and unmoved agents (one of them with contacts).

Plausible mistakes planted in the oracle (on the CPU) must trip at least one pin
(test_planted_mistakes_are_caught): in Eq. 1 (a dropped term, a sign, an index,
the radius), in the displacement (threshold, mass, dt, cap), in the grid
(padding, key order, scan) and in the adjoint (a sign, the cap projection, the
adherence mask, the pair Jacobian's transverse part).
"""
import dataclasses
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle import mech as M
from paper_2105_00039_gb300 import populations as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "eq1_worked_examples.json")


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


# ------------------------------------------------------------------ pin checks
def check_worked_examples():
    g = _golden()
    prm = O.Params(**g["params"])
    worst = 0.0
    for case in g["cases"]:
        st = np.array(case["state"], dtype=np.float64)
        r = O.step(st, prm, method="brute")
        worst = max(worst, float(np.abs(r["F"] - np.array(case["F"])).max()))
        if "u" in case:
            # the oracle uses the FP32 value of density 0.02 (2e-8 relative off)
            u = np.array(case["u"])
            rel = float(np.abs(r["u"] - u).max() / np.abs(u).max())
            worst = max(worst, 0.0 if rel < 1e-7 else rel)
    return worst


def _potential(pos, diam, prm):
    """Total pair potential; F = -grad E reproduces Eq. 1."""
    rad = 0.5 * diam
    I, J = O.pairs_bruteforce(pos, rad, prm.contact_margin)
    keep = I < J
    I, J = I[keep], J[keep]
    d = np.linalg.norm(pos[I] - pos[J], axis=1)
    delta = rad[I] + rad[J] + 2 * prm.contact_margin - d
    R = rad[I] * rad[J] / (rad[I] + rad[J])
    return float(np.sum(prm.k * delta ** 2 / 2 - (2.0 / 3.0) * prm.gamma * np.sqrt(R) * delta ** 1.5))


def _safe_cluster(n=24, seed=3, margin=0.0, side=None):
    """Random cluster with no pair within 2e-3 of the contact boundary."""
    for s in range(seed, seed + 200):
        side = side or 2.2 * n ** (1 / 3) * 5.0
        st = P.uniform_cube(n, side, 8.0, 12.0, s).astype(np.float64)
        pos, rad = st[:, :3], 0.5 * st[:, 3]
        d = np.linalg.norm(pos[:, None] - pos[None], axis=2)
        gap = rad[:, None] + rad[None] + 2 * margin - d
        np.fill_diagonal(gap, 1.0)
        if np.min(np.abs(gap)) > 2e-3 and (gap > 0).sum() >= n:
            return st
    raise RuntimeError("no safe cluster")


def check_potential_gradient(prm=O.Params(), n=24, seed=3):
    st = _safe_cluster(n, seed, prm.contact_margin)
    pos, diam = st[:, :3].copy(), st[:, 3]
    F = O.step(st, prm, method="brute")["F"]
    h = 1e-6
    G = np.zeros_like(pos)
    for i in range(n):
        for a in range(3):
            pp = pos.copy(); pp[i, a] += h
            pm = pos.copy(); pm[i, a] -= h
            G[i, a] = -(_potential(pp, diam, prm) - _potential(pm, diam, prm)) / (2 * h)
    return float(np.abs(G - F).max() / max(np.abs(F).max(), 1e-12))


def check_newton3(state, prm=O.Params()):
    r = O.step(state, prm)
    return float(np.abs(r["F"].sum(0)).max() / max(np.abs(r["F"]).sum(), 1e-300))


def check_pairs_methods_agree(state, margin=0.0):
    pos, rad = state[:, :3].astype(np.float64), 0.5 * state[:, 3].astype(np.float64)
    a = O.pairs_bruteforce(pos, rad, margin)
    b = O.pairs_kdtree(pos, rad, margin)
    return len(a[0]) == len(b[0]) and (a[0] == b[0]).all() and (a[1] == b[1]).all()


def check_grid_completeness(state32, margin=0.0):
    g = O.grid(state32, margin)
    pos, rad = state32[:, :3].astype(np.float64), 0.5 * state32[:, 3].astype(np.float64)
    I, J = O.pairs_bruteforce(pos, rad, margin)
    b = g["box"]
    ok = True
    ok &= bool(np.all(np.abs(b[I] - b[J]) <= 1))
    ok &= bool(np.all(b >= 1)) and bool(np.all(b <= g["dims"] - 2))
    ok &= int(g["start"][-1]) == len(state32)
    ok &= bool(np.all(np.diff(g["key"][g["perm"]]) >= 0))
    # each agent inside its box, allowing the FP32 rounding of (p - o)/e
    o = g["origin"].astype(np.float64)
    e = float(g["edge"])
    lo = o + b * e
    ok &= bool(np.all(pos >= lo - 1e-4 * e)) and bool(np.all(pos < lo + e + 1e-4 * e))
    return ok


def check_displacement_hand():
    """Worst relative deviation from hand-derived displacements (Sec. III rules
    as read here: strict adherence threshold, u = (dt / m) F with
    m = density (pi/6) d^3, cap to max_disp along u).  The parameters are
    float32-rounded by the oracle, hence the 1e-7 allowance."""
    worst = 0.0

    def rel(a, b):
        a, b = np.asarray(a, float), np.asarray(b, float)
        return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))

    # |F| = kappa delta = 0.5 exactly, threshold 0.5: no motion (strict >)
    r = O.step(np.array([[0, 0, 0, 10], [9.5, 0, 0, 10]], float),
               O.Params(k=1.0, gamma=0.0, adherence=0.5), method="brute")
    worst = max(worst, float(np.abs(r["u"]).max()))
    # deep overlap (phi = 10 - sqrt(12.5)), dt = 1/2, d = 10: m = 0.02 pi/6 1000
    deep = np.array([[0, 0, 0, 10], [0, 5, 0, 10]], float)
    u_half = 0.5 * (10.0 - math.sqrt(12.5)) / (0.02 * math.pi / 6.0 * 1000.0)   # 0.30866
    r = O.step(deep, O.Params(dt=0.5), method="brute")
    worst = max(worst, rel(r["u"], [[0, -u_half, 0], [0, u_half, 0]]))
    # the same with max_disp 0.2 < 0.30866: |u| = 0.2 along the same line
    r = O.step(deep, O.Params(dt=0.5, max_disp=0.2), method="brute")
    worst = max(worst, rel(r["u"], [[0, -0.2, 0], [0, 0.2, 0]]))
    # a d = 20 sphere against a d = 10 one with delta = 1 and gamma = 0: |F| = 1,
    # m = 0.02 pi/6 8000, so |u| = 1/(0.02 pi/6 8000) for the large one
    r = O.step(np.array([[0, 0, 0, 20], [14, 0, 0, 10]], float),
               O.Params(k=1.0, gamma=0.0, adherence=0.0), method="brute")
    worst = max(worst, rel(r["u"][0], [-1.0 / (0.02 * math.pi / 6.0 * 8000.0), 0, 0]))
    return 0.0 if worst < 1e-7 else worst


def check_grid_hand():
    """Two d = 10 spheres at x = 0 and x = 25: edge 10 + 8 ulp(25) = 10 + 2^-16,
    one empty padding layer, so boxes (1,1,1) and (3,1,1) of a 5x3x3 grid,
    x-fastest keys 21 and 23, starts 0 | 1 | 2 around them."""
    g = O.grid(np.array([[0, 0, 0, 10], [25, 0, 0, 10]], dtype=np.float32))
    e = np.float32(10.0 + 2.0 ** -16)
    return bool(g["edge"] == e and np.array_equal(g["origin"], [-e, -e, -e])
                and list(g["dims"]) == [5, 3, 3] and list(g["key"]) == [21, 23]
                and g["nboxes"] == 45 and list(g["perm"]) == [0, 1]
                and list(g["start"][20:25]) == [0, 0, 1, 1, 2] and g["start"][-1] == 2)


def check_grid_slices_hand():
    """The order inside a box (the library's reading; the paper fixes none).
    44 spheres of d = 10 in one box, x cycling through 9, 1, 7, 3: the grid is
    3x3x3 = 27 boxes, so 4 * 2 * 27 = 216 <= 5 * 44 = 220 gives K = 2 slices
    (K = 4 would need 432 <= 220).  With o = 1 - e, t_x = 1 + (x - 1) / e puts
    x = 1, 3 in slice 0 and x = 7, 9 in slice 1 (fractions 0, 0.2, 0.6, 0.8), so
    the sorted order is every x = 1 or 3 agent (the odd input indices) in input
    order, then the x = 7 or 9 ones (the even indices); 43 agents give K = 1
    and plain input order."""
    x = np.array([[9, 0, 0, 10], [1, 0, 0, 10], [7, 0, 0, 10], [3, 0, 0, 10]] * 11, np.float32)
    g = O.grid(x)
    ok = g["ks"] == 1 and g["nboxes"] == 27 and list(g["sub"][:4]) == [1, 0, 1, 0]
    ok &= list(g["perm"]) == list(range(1, 44, 2)) + list(range(0, 44, 2))
    # the slice table: box 13 (the middle one) holds 22 + 22 agents
    ok &= list(g["table"][26:29]) == [0, 22, 44] and g["table"][-1] == 44
    g43 = O.grid(x[:43])
    ok &= g43["ks"] == 0 and list(g43["perm"]) == list(range(43))
    return bool(ok)


def check_grid_slice_order(state32, margin=0.0):
    """Sorted agents of every box come by slice, then by input index, and the
    slice table counts them."""
    g = O.grid(state32, margin)
    K = 1 << g["ks"]
    perm = g["perm"]
    sk = g["key"][perm] * K + g["sub"][perm]
    ok = bool(np.all(np.diff(sk) >= 0))
    same = np.diff(sk) == 0
    ok &= bool(np.all(np.diff(perm)[same] > 0))
    # a slice spans 1/K of its box along x
    o, e = g["origin"].astype(np.float64), float(g["edge"])
    fx = (state32[:, 0].astype(np.float64) - o[0]) / e - g["box"][:, 0]
    ok &= bool(np.all(fx >= g["sub"] / K - 1e-5)) and bool(np.all(fx < (g["sub"] + 1) / K + 1e-5))
    ok &= bool(np.array_equal(np.diff(g["table"]), np.bincount(g["key"] * K + g["sub"],
                                                              minlength=K * g["nboxes"])))
    return ok


# ------------------------------------------------------------------ tests
def test_sub_bin_rule_values():
    """4 * 2^ks * nboxes <= 5 * n, ks <= 3: thresholds worked by hand for 27 boxes."""
    assert [O.sub_bin_shift(n, 27) for n in (0, 43, 44, 86, 87, 172, 173, 10 ** 6)] == \
        [0, 0, 1, 1, 2, 2, 3, 3]
    assert O.sub_bin_shift(10, 0) == 0


def test_windowed_walk_test_populations_use_1_to_8_slices():
    """The populations that tests/test_gpu_windows.py walks both ways cover
    every number of x slices per box."""
    from test_gpu_windows import _cases
    ks = {name: O.grid(st, m)["ks"] for name, (st, m) in _cases().items()}
    assert {ks["sparse_K1"], ks["lattice_K2"], ks["dense_K4"], ks["dense_K8"]} == {0, 1, 2, 3}


def test_grid_slices_hand_example():
    assert check_grid_slices_hand()


@pytest.mark.parametrize("seed", [0, 1])
def test_grid_slice_order(seed):
    assert check_grid_slice_order(P.small_uniform(seed))
    assert check_grid_slice_order(P.uniform_cube(3000, 60.0, 8.0, 12.0, seed))        # K = 4
    assert check_grid_slice_order(P.jittered_lattice(4096, 16, 9.0, 1.5, 9.0, 11.0, seed), 1.5)
    assert O.grid(P.uniform_cube(3000, 60.0, 8.0, 12.0, seed))["ks"] >= 2


def test_worked_examples():
    assert check_worked_examples() < 1e-12


def test_force_is_minus_potential_gradient():
    assert check_potential_gradient() < 1e-7


def test_force_is_minus_potential_gradient_with_margin_and_constants():
    assert check_potential_gradient(O.Params(k=2.5, gamma=1.2, contact_margin=0.75), n=20, seed=11) < 1e-7


@pytest.mark.parametrize("seed", [0, 1])
def test_newton_third_law(seed):
    assert check_newton3(P.small_uniform(seed)) < 1e-13


def test_non_overlapping_contribute_nothing():
    st = P.jittered_lattice(64, 4, 13.0, 0.4, 8.0, 12.0, seed=2)   # gaps >= 13 - 0.8 - 12 > 0
    r = O.step(st, O.Params())
    assert len(r["I"]) == 0 and np.all(r["F"] == 0) and np.all(r["u"] == 0)


def test_self_pair_and_coincident_centres():
    st = np.array([[1, 2, 3, 10], [1, 2, 3, 10], [8, 2, 3, 10]], dtype=np.float32)
    r = O.step(st, O.Params(), method="brute")
    pairs = set(zip(r["I"].tolist(), r["J"].tolist()))
    assert pairs == {(0, 2), (2, 0), (1, 2), (2, 1)}   # coincident pair (0, 1) excluded
    assert np.all(np.isfinite(r["F"]))


def test_rotation_and_axis_permutation_invariance():
    st = P.small_uniform(4)[:1500].astype(np.float64)
    r0 = O.step(st, O.Params())
    perm = [2, 0, 1]
    st2 = st.copy(); st2[:, :3] = st[:, perm]
    r1 = O.step(st2, O.Params())
    assert np.array_equal(r0["I"], r1["I"])
    np.testing.assert_allclose(r1["F"], r0["F"][:, perm], rtol=0, atol=1e-12)
    th = 0.7
    Q = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    st3 = st.copy(); st3[:, :3] = st[:, :3] @ Q.T
    r3 = O.step(st3, O.Params(), pairs=(r0["I"], r0["J"]))
    np.testing.assert_allclose(r3["F"], r0["F"] @ Q.T, rtol=0, atol=1e-10)


def test_input_permutation_invariance():
    st = P.small_uniform(5)[:2000]
    rng = np.random.default_rng(0)
    q = rng.permutation(len(st))
    r0 = O.step(st, O.Params())
    r1 = O.step(st[q], O.Params())
    np.testing.assert_allclose(r1["F"], r0["F"][q], rtol=0, atol=1e-12)
    np.testing.assert_allclose(r1["u"], r0["u"][q], rtol=0, atol=1e-13)


def test_length_scaling():
    # phi(lambda delta; lambda R) = lambda phi: all lengths x2 doubles F
    st = P.small_uniform(6)[:1000].astype(np.float64)
    r0 = O.step(st, O.Params())
    r1 = O.step(2 * st, O.Params())
    np.testing.assert_allclose(r1["F"], 2 * r0["F"], rtol=0, atol=1e-11)


@pytest.mark.parametrize("kind", ["uniform", "lattice", "clustered"])
def test_kdtree_equals_bruteforce(kind):
    if kind == "uniform":
        st = P.small_uniform(7)
    elif kind == "lattice":
        st = P.jittered_lattice(4096, 16, 9.0, 1.5, 9.0, 11.0, 7)
    else:
        st = P.uniform_cube(3000, 60.0, 8.0, 12.0, 7)      # ~50 neighbours each
    assert check_pairs_methods_agree(st)
    assert check_pairs_methods_agree(st, margin=1.5)


def test_pair_count_small_lattice():
    # 2x2x2 lattice, spacing 9, d = 10: each agent touches its 3 face neighbours
    st = P.jittered_lattice(8, 2, 9.0, 0.0, 10.0, 10.0, 0)
    I, J = O.pairs_bruteforce(st[:, :3].astype(float), 0.5 * st[:, 3].astype(float))
    assert len(I) == 24


def test_grid_hand_example():
    # S = 10, C = 25: ulp(25) = 2^-19, edge = 10 + 8 * 2^-19 = 10 + 2^-16
    assert check_grid_hand()


def test_displacement_hand_values():
    assert check_displacement_hand() == 0.0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_grid_completeness(seed):
    assert check_grid_completeness(P.small_uniform(seed))
    assert check_grid_completeness(P.jittered_lattice(4096, 16, 9.0, 1.5, 9.0, 11.0, seed), 1.5)
    assert check_grid_completeness(P.uniform_cube(2000, 40.0, 8.0, 12.0, seed))


def test_grid_edge_margin_keeps_face_pairs_adjacent():
    # two maximal spheres just touching across a box face far from the origin:
    # the box edge's rounding margin keeps them in adjacent boxes
    x0 = np.float32(4096.0)
    st = np.array([[x0, 0, 0, 10], [np.nextafter(x0 + 10, np.float32(0)), 0, 0, 10]], np.float32)
    g = O.grid(st)
    assert g["edge"] > 10 and abs(int(g["box"][0, 0]) - int(g["box"][1, 0])) <= 1
    assert check_grid_completeness(st)


def test_grid_negative_and_tiny_extent():
    st = np.array([[-5.5, -100, 3, 9], [-5.25, -100, 3, 11]], dtype=np.float32)
    assert check_grid_completeness(st)
    g = O.grid(st)
    assert list(g["dims"]) == [3, 3, 3]


def test_displacement_rules():
    prm = O.Params(k=1.0, gamma=0.0, adherence=0.5, max_disp=3.0)
    st = np.array([[0, 0, 0, 10], [9.5, 0, 0, 10]], dtype=np.float64)   # delta = 0.5, |F| = 0.5
    r = O.step(st, prm, method="brute")
    assert np.all(r["Fn"] == 0.5) and not r["moving"].any()            # strict >
    r = O.step(st, O.Params(k=1.0, gamma=0.0, adherence=0.4999, max_disp=3.0), method="brute")
    assert r["moving"].all()
    # cap: |v| = 6.4645/10.47 = 0.617 > 0.5 -> |u| = 0.5, direction kept
    st = np.array([[0, 0, 0, 10], [0, 5, 0, 10]], dtype=np.float64)
    r = O.step(st, O.Params(max_disp=0.5), method="brute")
    np.testing.assert_allclose(np.linalg.norm(r["u"], axis=1), 0.5, rtol=1e-15)
    np.testing.assert_allclose(r["u"][0] / 0.5, [0, -1, 0], atol=1e-15)
    r = O.step(st, O.Params(max_disp=0.7), method="brute")
    assert not r["capped"].any()
    # freeze (benchmark B rule): max displacement 0
    r = O.step(P.small_uniform(0), O.Params(max_disp=0.0))
    assert np.all(r["u"] == 0)


def test_mass_scaling_of_displacement():
    # same force, diameter doubled -> displacement / 8 (m ~ d^3)
    prm = O.Params(k=1.0, gamma=0.0, adherence=0.0)
    a = O.step(np.array([[0, 0, 0, 10], [9, 0, 0, 10]], float), prm, method="brute")
    # a sphere of d=20 against a d=0.0 ... use a contact with the same delta
    b = O.step(np.array([[0, 0, 0, 20], [14, 0, 0, 10]], float), prm, method="brute")
    assert a["F"][0, 0] == b["F"][0, 0] == -1.0
    np.testing.assert_allclose(b["u"][0, 0] * 8, a["u"][0, 0], rtol=1e-14)


# ------------------------------------------------------------------ adjoint pins
def _fd_fixture(seed=5, n=27, steps=3, still_contact=False):
    """A 3x3x3 jittered lattice whose trajectory keeps every piecewise test
    (adherence, cap, contact onset) far from its boundary, with capped and
    unmoved agents; with still_contact=True an unmoved agent that has contacts
    (its force below the adherence threshold but not zero) in every step."""
    for s in range(seed, seed + 300):
        st = P.jittered_lattice(n, 3, 9.0, 1.5, 9.0, 11.0, s).astype(np.float64)
        prm = O.Params(adherence=0.05, max_disp=0.045)
        _, recs = O.trajectory(st, prm, steps, "brute", keep=True)
        ok = True
        for rec in recs:
            mg = O.margins(rec, prm)
            pos, rad = rec["state"][:, :3], 0.5 * rec["state"][:, 3]
            d = np.linalg.norm(pos[:, None] - pos[None], axis=2)
            gap = rad[:, None] + rad[None] - d
            np.fill_diagonal(gap, 1.0)
            ok &= mg["adherence"].min() > 1e-4 and mg["cap"].min() > 1e-4
            ok &= np.abs(gap).min() > 2e-3
        if still_contact:
            ok &= all(((~r["moving"]) & (r["npairs"] > 0)).any() for r in recs)
        if ok and any(r["capped"].any() for r in recs) and any((~r["moving"]).any() for r in recs):
            return st, prm
    raise RuntimeError("no FD-safe fixture")


def check_adjoint_fd(steps=3, still_contact=False):
    st, prm = _fd_fixture(steps=steps, still_contact=still_contact)
    n = len(st)
    target = st[:, :3] + 0.3 * np.sin(np.arange(3 * n).reshape(n, 3))
    res = O.trajectory_grad(st, target, prm, steps, "brute")
    h = 1e-6
    errs = []

    def L(state=st, p=prm):
        return O.trajectory_loss(state, target, p, steps, "brute")

    for name, key in (("k", "dk"), ("gamma", "dgamma")):
        pp = O.Params(**{**prm.__dict__}); setattr(pp, name, getattr(prm, name) + h)
        pm = O.Params(**{**prm.__dict__}); setattr(pm, name, getattr(prm, name) - h)
        # the oracle rounds params to FP32; perturb in FP64 by bypassing that
        fd = (_loss64(st, target, pp, steps) - _loss64(st, target, pm, steps)) / (2 * h)
        errs.append(abs(fd - res[key]) / max(abs(fd), 1e-12))
    rng = np.random.default_rng(1)
    for _ in range(3):
        dirn = np.zeros_like(st)
        dirn[:, :3] = rng.standard_normal((n, 3))
        dirn[:, 3] = 0.3 * rng.standard_normal(n)
        fd = (L(st + h * dirn) - L(st - h * dirn)) / (2 * h)
        an = float(np.sum(res["dpos"] * dirn[:, :3]) + np.sum(res["ddiam"] * dirn[:, 3]))
        errs.append(abs(fd - an) / max(abs(fd), 1e-12))
    return max(errs)


def _loss64(st, target, prm, steps):
    """Loss with parameters used at full FP64 (no FP32 rounding), for FD in k, gamma."""
    orig = M.Params.as64
    try:
        M.Params.as64 = lambda self: self
        return O.trajectory_loss(st, target, prm, steps, "brute")
    finally:
        M.Params.as64 = orig


@pytest.mark.parametrize("still_contact", [False, True])
def test_adjoint_matches_central_differences(still_contact):
    orig = M.Params.as64
    try:
        M.Params.as64 = lambda self: self      # FD in FP64 parameters on both sides
        assert check_adjoint_fd(still_contact=still_contact) < 1e-6
    finally:
        M.Params.as64 = orig


# ------------------------------------------------------------------ planted mistakes
def _plant(monkeypatch, which):
    orig_terms = M.pair_terms
    orig_disp = M.displacement
    orig_grad = M.trajectory_grad

    if which == "drop_gamma":
        def terms(pos, diam, prm, I, J):
            t = orig_terms(pos, diam, prm, I, J)
            t["phi"] = prm.k * t["delta"]
            return t
        monkeypatch.setattr(M, "pair_terms", terms)
    elif which == "wrong_sign":
        def terms(pos, diam, prm, I, J):
            t = orig_terms(pos, diam, prm, I, J)
            t["u"] = -t["u"]
            return t
        monkeypatch.setattr(M, "pair_terms", terms)
    elif which == "diameter_as_radius":
        def terms(pos, diam, prm, I, J):
            return orig_terms(pos, 2.0 * diam, prm, I, J)
        monkeypatch.setattr(M, "pair_terms", terms)
    elif which == "R_sum":
        def terms(pos, diam, prm, I, J):
            t = orig_terms(pos, diam, prm, I, J)
            r = 0.5 * diam
            R = r[I] + r[J]
            t["root"] = np.sqrt(R * t["delta"])
            t["phi"] = prm.k * t["delta"] - prm.gamma * t["root"]
            return t
        monkeypatch.setattr(M, "pair_terms", terms)
    elif which == "transposed_index":
        def terms(pos, diam, prm, I, J):
            return orig_terms(pos, diam, prm, J, I)
        monkeypatch.setattr(M, "pair_terms", terms)
    elif which == "adherence_ge":
        def disp(F, diam, prm):
            r = orig_disp(F, diam, prm)
            mv = r["Fn"] >= prm.adherence
            r["moving"] = mv
            r["u"] = np.where(mv[:, None], r["v"], 0.0)
            return r
        monkeypatch.setattr(M, "displacement", disp)
    elif which == "mass_from_radius":
        monkeypatch.setattr(M, "mass", lambda diam, prm: prm.density * (np.pi / 6.0) * (0.5 * diam) ** 3)
    elif which == "dt_ignored":
        monkeypatch.setattr(M, "displacement",
                            lambda F, diam, prm: orig_disp(F, diam, dataclasses.replace(prm, dt=1.0)))
    elif which == "cap_ignored":
        monkeypatch.setattr(M, "displacement",
                            lambda F, diam, prm: orig_disp(F, diam, dataclasses.replace(prm, max_disp=np.inf)))
    elif which.startswith("grid_"):
        orig_grid = M.grid

        def grid(state32, contact_margin=0.0):
            g = dict(orig_grid(state32, contact_margin))
            b, dims = g["box"].copy(), g["dims"].copy()
            if which == "grid_no_padding":          # origin at the minimum, no empty layer
                b, dims = b - 1, dims - 1
            if which == "grid_key_y_fastest":
                key = (b[:, 2] * dims[0] + b[:, 0]) * dims[1] + b[:, 1]
            else:
                key = (b[:, 2] * dims[1] + b[:, 1]) * dims[0] + b[:, 0]
            nboxes = int(np.prod(dims))
            counts = np.bincount(key, minlength=nboxes)
            start = np.zeros(nboxes + 1, dtype=np.int64)
            if which == "grid_inclusive_scan":
                start[:-1] = np.cumsum(counts)
                start[-1] = start[-2]
            else:
                start[1:] = np.cumsum(counts)
            ks, sub = g["ks"], g["sub"]
            if which == "grid_slices_doubled":      # one more slice level than the rule gives
                ks = ks + 1
                sub = np.minimum(np.floor(((state32[:, 0] - g["origin"][0]) / g["edge"]).astype(np.float32)
                                          - b[:, 0]) * (1 << ks), (1 << ks) - 1).astype(np.int64)
            K = 1 << ks
            skey = key * K + sub
            perm = np.argsort(key if which == "grid_box_input_order" else skey, kind="stable")
            table = np.zeros(K * nboxes + 1, dtype=np.int64)
            table[1:] = np.cumsum(np.bincount(skey, minlength=K * nboxes))
            g.update(box=b, dims=dims, key=key, nboxes=nboxes, counts=counts, start=start,
                     ks=ks, sub=sub, table=table, perm=perm)
            return g
        monkeypatch.setattr(M, "grid", grid)
        monkeypatch.setattr(O, "grid", grid)


def _pins_pass(which):
    g_ok = check_worked_examples() < 1e-12
    p_ok = check_potential_gradient(n=16, seed=3) < 1e-7
    n_ok = check_newton3(P.small_uniform(0)[:1500]) < 1e-13
    d_ok = check_displacement_hand() == 0.0
    b_ok = check_grid_hand() and check_grid_completeness(P.small_uniform(0))
    b_ok = b_ok and check_grid_slices_hand()
    return g_ok and p_ok and n_ok and d_ok and b_ok


@pytest.mark.parametrize("which", ["drop_gamma", "wrong_sign", "diameter_as_radius", "R_sum",
                                   "transposed_index", "adherence_ge", "mass_from_radius",
                                   "dt_ignored", "cap_ignored", "grid_no_padding",
                                   "grid_key_y_fastest", "grid_inclusive_scan",
                                   "grid_box_input_order", "grid_slices_doubled"])
def test_planted_mistakes_are_caught(monkeypatch, which):
    assert _pins_pass("none")
    _plant(monkeypatch, which)
    assert not _pins_pass(which)


def test_planted_adjoint_mistake_is_caught(monkeypatch):
    orig = M.trajectory_grad

    def bad(*a, **k):
        r = orig(*a, **k)
        r["dk"] = -r["dk"]
        return r
    monkeypatch.setattr(M.Params, "as64", lambda self: self)
    assert check_adjoint_fd() < 1e-6
    monkeypatch.setattr(O, "trajectory_grad", bad)
    assert check_adjoint_fd() > 1e-3


@pytest.mark.parametrize("which", ["cap_branch_dropped", "adherence_branch_dropped",
                                   "transverse_term_dropped"])
def test_planted_reverse_pass_mistakes_are_caught(monkeypatch, which):
    """Mistakes inside the reverse pass, planted through the forward records it
    reads (the forward trajectory and the loss are untouched): the cap's
    projection or the adherence mask forgotten, or the pair Jacobian without
    its (phi/d)(I - u u^T) part."""
    monkeypatch.setattr(M.Params, "as64", lambda self: self)
    assert check_adjoint_fd(still_contact=True) < 1e-6
    orig = M.trajectory

    def traj(state0, prm=O.Params(), nsteps=1, method="auto", keep=False):
        out = orig(state0, prm, nsteps, method, keep)
        if not keep:
            return out
        final, recs = out
        for r in recs:
            if which == "cap_branch_dropped":
                r["capped"] = np.zeros_like(r["capped"])
            elif which == "adherence_branch_dropped":
                r["moving"] = np.ones_like(r["moving"])
            else:
                r["terms"] = dict(r["terms"], phi=np.zeros_like(r["terms"]["phi"]))
        return final, recs
    monkeypatch.setattr(M, "trajectory", traj)
    assert check_adjoint_fd(still_contact=True) > 1e-3


def test_sampled_form_equals_full_step():
    st = P.jittered_lattice(4096, 16, 9.0, 1.5, 9.0, 11.0, 3)
    prm = O.Params(contact_margin=0.5)
    full = O.step(st, prm, method="brute")
    idx = np.arange(0, 4096, 7)
    smp = O.step_sampled(st, idx, prm)
    np.testing.assert_allclose(smp["F"], full["F"][idx], rtol=0, atol=1e-12)
    np.testing.assert_allclose(smp["u"], full["u"][idx], rtol=0, atol=1e-13)
    assert np.array_equal(smp["npairs"], full["npairs"][idx])


def test_reverse_pass_along_own_states_is_the_same():
    st, prm = _fd_fixture(steps=3)
    n = len(st)
    target = st[:, :3] + 0.2
    ref = O.trajectory_grad(st, target, prm, 3, "brute")
    _, recs = O.trajectory(st, prm, 3, "brute", keep=True)
    states = [r["state"] for r in recs] + [ref["final"]]
    alt = O.trajectory_grad_along(states, target, prm, "brute")
    assert alt["dk"] == ref["dk"] and alt["dgamma"] == ref["dgamma"]
    assert np.array_equal(alt["dpos"], ref["dpos"]) and np.array_equal(alt["ddiam"], ref["ddiam"])
