"""The library's adjoint (ug_step_backward behind a torch.autograd.Function)
against the FP64 oracle's adjoint and against FP64 central differences."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2105_00039_gb300 import populations as P

from _metrics import record

pytestmark = pytest.mark.gpu
DEV = "cuda"
TOL = 1e-3


@pytest.fixture(scope="module")
def U():
    from paper_2105_00039_gb300 import ugmech
    ugmech.load()
    return ugmech


def _gpu_grad(U, st, target, prm_u, steps, ckpt):
    from paper_2105_00039_gb300.autograd import trajectory
    x = torch.from_numpy(np.ascontiguousarray(st, np.float32)).to(DEV).requires_grad_(True)
    k = torch.tensor(float(prm_u.k), requires_grad=True)
    g = torch.tensor(float(prm_u.gamma), requires_grad=True)
    out = trajectory(x, k, g, prm_u, steps, ckpt)
    tgt = torch.from_numpy(np.asarray(target, np.float64)).to(DEV)
    loss = ((out[:, :3].double() - tgt) ** 2).mean()
    loss.backward()
    return (float(loss.detach()), float(k.grad), float(g.grad), x.grad[:, :3].double().cpu().numpy(),
            x.grad[:, 3].double().cpu().numpy())


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-30)


def _nrel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _fd64(fn, x, h):
    import oracle.mech as M
    orig = M.Params.as64
    try:
        M.Params.as64 = lambda self: self        # perturb parameters in FP64
        return (fn(x + h) - fn(x - h)) / (2 * h)
    finally:
        M.Params.as64 = orig


def test_adjoint_small_with_adherence_and_cap(U):
    """A fixture whose trajectory stays clear of every piecewise boundary
    (adherence, cap, contact onset): GPU gradient = oracle adjoint = FP64 central
    differences with h = 1e-3."""
    from test_oracle_pins import _fd_fixture
    st, prm = _fd_fixture(steps=3)
    n = len(st)
    target = st[:, :3] + 0.3 * np.sin(np.arange(3 * n).reshape(n, 3))
    st32 = st.astype(np.float32)
    ref = O.trajectory_grad(st32, target, prm, 3, "brute")
    prm_u = U.Params(adherence=prm.adherence, max_disp=prm.max_disp)
    L, dk, dg, dp, dd = _gpu_grad(U, st32, target, prm_u, 3, 2)
    assert _rel(L, ref["loss"]) < 1e-5
    assert _rel(dk, ref["dk"]) < TOL and _rel(dg, ref["dgamma"]) < TOL
    assert _nrel(dp, ref["dpos"]) < TOL and _nrel(dd, ref["ddiam"]) < TOL
    s64 = st32.astype(np.float64)
    mk = lambda k: O.Params(k=k, adherence=prm.adherence, max_disp=prm.max_disp)
    mg = lambda g: O.Params(gamma=g, adherence=prm.adherence, max_disp=prm.max_disp)
    fk = _fd64(lambda k: O.trajectory_loss(s64, target, mk(k), 3, "brute"), 2.0, 1e-3)
    fg = _fd64(lambda g: O.trajectory_loss(s64, target, mg(g), 3, "brute"), 1.0, 1e-3)
    assert _rel(dk, fk) < TOL and _rel(dg, fg) < TOL, (dk, fk, dg, fg)
    v = P.random_unit_vectors(n, seed=4)
    fd = _fd64(lambda a: O.trajectory_loss(np.concatenate([s64[:, :3] + a * v, s64[:, 3:]], 1),
                                           target, prm, 3, "brute"), 0.0, 1e-3)
    assert _rel(float(np.sum(dp * v)), fd) < TOL


def test_adjoint_unmoved_agent_in_contact(U):
    """Adherence with contacts: in every step an agent touches others while
    its force stays below the threshold, so the reverse pass must stop at it
    (no displacement, no force sensitivity) yet keep its neighbours' pair
    terms.  GPU gradient = FP64 oracle adjoint on the same float32 rows."""
    from test_oracle_pins import _fd_fixture
    st, prm = _fd_fixture(steps=3, still_contact=True)
    n = len(st)
    target = st[:, :3] + 0.3 * np.sin(np.arange(3 * n).reshape(n, 3))
    st32 = st.astype(np.float32)
    _, recs = O.trajectory(st32, prm, 3, "brute", keep=True)
    assert all(((~r["moving"]) & (r["npairs"] > 0)).any() for r in recs)
    ref = O.trajectory_grad(st32, target, prm, 3, "brute")
    prm_u = U.Params(adherence=prm.adherence, max_disp=prm.max_disp)
    L, dk, dg, dp, dd = _gpu_grad(U, st32, target, prm_u, 3, 2)
    assert _rel(L, ref["loss"]) < 1e-5
    assert _rel(dk, ref["dk"]) < TOL and _rel(dg, ref["dgamma"]) < TOL
    assert _nrel(dp, ref["dpos"]) < TOL and _nrel(dd, ref["ddiam"]) < TOL


def _lattice_case(side, steps):
    st = P.lattice_cube(side, seed=5)
    prm_t = O.Params(k=2.5, gamma=1.2, adherence=0.0)
    target = O.trajectory(st, prm_t, steps)[:, :3]          # FP64 target trajectory
    return st, target


def _gpu_states(U, st, prm_u, steps):
    x = torch.from_numpy(st).to(DEV)
    n = len(st)
    sp = U.Stepper(n, U.estimate_max_boxes(x, prm_u.contact_margin, slack=3.0), x.device)
    perm = U.iota(n, x.device)
    states = [st.astype(np.float64)]
    for _ in range(steps):
        sp.step(x, perm, prm_u, 1)
        states.append(U.scatter_rows(x, perm).cpu().numpy().astype(np.float64))
    sp.check()
    return states


def test_adjoint_lattice_along_gpu_trajectory(U):
    """The differentiable workload's recipe on a 16^3 lattice: 50 steps,
    checkpoints every 10, target from kappa=2.5, gamma=1.2, gradients at
    kappa=2, gamma=1.  The loss has kinks wherever a pair touches (sqrt(delta)),
    so the float32 and FP64 trajectories may cross different kinks; the oracle's
    adjoint is therefore evaluated along the GPU's own trajectory."""
    steps = 50
    st, target = _lattice_case(16, steps)
    prm = O.Params(adherence=0.0)
    L, dk, dg, dp, dd = _gpu_grad(U, st, target, U.Params(adherence=0.0), steps, 10)
    states = _gpu_states(U, st, U.Params(adherence=0.0), steps)
    ref = O.trajectory_grad_along(states, target, prm)
    assert _rel(L, ref["loss"]) < 1e-6
    assert _rel(dk, ref["dk"]) < TOL, (dk, ref["dk"])
    assert _rel(dg, ref["dgamma"]) < TOL, (dg, ref["dgamma"])
    assert _nrel(dp, ref["dpos"]) < TOL
    assert _nrel(dd, ref["ddiam"]) < TOL


def test_adjoint_full_size_along_gpu_trajectory(U):
    """The differentiable configuration at full size (64^3 cells, 50 steps,
    checkpoints every 10): GPU gradients against the FP64 oracle adjoint along
    the GPU's own trajectory (about a minute of oracle time)."""
    steps = 50
    st, target = _lattice_case(64, steps)
    L, dk, dg, dp, dd = _gpu_grad(U, st, target, U.Params(adherence=0.0), steps, 10)
    states = _gpu_states(U, st, U.Params(adherence=0.0), steps)
    ref = O.trajectory_grad_along(states, target, O.Params(adherence=0.0), "kdtree")
    record("dL/dkappa (64^3 cells, 50 steps; oracle adjoint along the GPU trajectory)",
           rel=_rel(dk, ref["dk"]), gpu=dk, oracle=ref["dk"], tolerance=TOL)
    record("dL/dgamma (64^3 cells, 50 steps; oracle adjoint along the GPU trajectory)",
           rel=_rel(dg, ref["dgamma"]), gpu=dg, oracle=ref["dgamma"], tolerance=TOL)
    ep = np.linalg.norm(dp - ref["dpos"], axis=1) / max(np.linalg.norm(ref["dpos"], axis=1).max(), 1e-30)
    record("dL/dp (64^3 cells, 50 steps; oracle adjoint along the GPU trajectory)",
           normwise=_nrel(dp, ref["dpos"]), max_row_over_largest=ep.max(), median_row_over_largest=np.median(ep),
           tolerance=TOL)
    record("dL/d(diameter) (64^3 cells, 50 steps; oracle adjoint along the GPU trajectory)",
           normwise=_nrel(dd, ref["ddiam"]), tolerance=TOL)
    assert _rel(dk, ref["dk"]) < TOL and _rel(dg, ref["dgamma"]) < TOL
    assert _nrel(dp, ref["dpos"]) < TOL
    assert _nrel(dd, ref["ddiam"]) < TOL


def test_adjoint_full_size_beside_finite_differences(U):
    """The differentiable configuration's gradients in k and gamma beside FP64
    central differences of the oracle's loss at h = 3e-3, 1e-3 and 3e-4 and the
    oracle's adjoint along its own FP64 trajectory (tests/golden/fd_lattice64.json,
    written by the oracle alone).  sqrt(delta) puts a kink into the loss
    wherever a pair starts or stops touching, and 262,144 cells over 50 steps
    cross many of them, so central differences measure the kinks' jumps as well
    as the slope: they move with h and sit a few per cent from the adjoint.
    The GPU's gradient must agree with the oracle adjoint (its float32
    trajectory crosses slightly different kinks: 2e-2) and lie no farther from
    the differences than the oracle adjoint itself does (plus that 2e-2)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "fd_lattice64.json")) as f:
        gold = json.load(f)
    steps = 50
    st, target = _lattice_case(64, steps)
    L, dk, dg, dp, dd = _gpu_grad(U, st, target, U.Params(adherence=0.0), steps, 10)
    adj = gold["oracle_adjoint"]
    rk, rg = _rel(dk, adj["dL_dkappa"]), _rel(dg, adj["dL_dgamma"])
    for fd in gold["central_differences"]:
        gk, gg = _rel(dk, fd["dL_dkappa"]), _rel(dg, fd["dL_dgamma"])
        ok_k, ok_g = _rel(adj["dL_dkappa"], fd["dL_dkappa"]), _rel(adj["dL_dgamma"], fd["dL_dgamma"])
        record(f"dL/dkappa, dL/dgamma vs FP64 central differences, h = {fd['h']} (64^3 cells, 50 steps)",
               gpu_kappa=dk, fd_kappa=fd["dL_dkappa"], rel_kappa=gk, oracle_adjoint_rel_kappa=ok_k,
               gpu_gamma=dg, fd_gamma=fd["dL_dgamma"], rel_gamma=gg, oracle_adjoint_rel_gamma=ok_g)
        assert gk <= ok_k + 2e-2 and gg <= ok_g + 2e-2
    record("dL/dkappa, dL/dgamma vs the oracle adjoint along its own FP64 trajectory (64^3, 50 steps)",
           rel_kappa=rk, rel_gamma=rg, loss_gpu=L, loss_oracle=gold["loss"])
    assert rk < 2e-2 and rg < 2e-2
    assert _rel(L, gold["loss"]) < 1e-3


def test_backward_is_deterministic_and_zero_steps(U):
    st = P.lattice_cube(10, seed=2)
    x = torch.from_numpy(st).to(DEV)
    mb = U.estimate_max_boxes(x, 0.0, slack=3.0)
    G = torch.randn(len(st), 4, device=DEV)
    a, ga, s1 = U.step_backward(x, U.Params(), 4, mb, G)
    b, gb, s2 = U.step_backward(x, U.Params(), 4, mb, G)
    U.check_status(s1)
    U.check_status(s2)
    assert torch.equal(a, b) and torch.equal(ga, gb)
    c, gc, _ = U.step_backward(x, U.Params(), 0, mb, G)
    assert torch.equal(c, G) and float(gc.abs().sum()) == 0.0
