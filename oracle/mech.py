"""FP64 CPU oracle for one mechanical-interaction step of spherical agents.

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg may import this package.  It shares no code with
the CUDA library and never calls it.

What it computes (Hesam et al., "GPU Acceleration of 3D Agent-Based Biological
Simulations", Sec. III, Eq. 1 and the paragraph after it; Sec. IV-A for the grid):

  for every ordered pair (i, j), i != j (self excluded by index):
      d     = ||p_i - p_j||
      delta = r_i + r_j + 2m - d                        (Eq. 1, first line; m = contact margin)
      if delta > 0 and d > 0:
          R   = r_i r_j / (r_i + r_j)                    (Eq. 1, second line; true radii)
          phi = kappa * delta - gamma * sqrt(R * delta)  (Eq. 1, third line)
          f_ij = phi * (p_i - p_j) / d
  F_i = sum_j f_ij

  Displacement (Sec. III; the paper names the three stages but gives no formula,
  so these are the readings this library fixes):
      mass      m_i = rho * (pi / 6) * d_i^3
      adherence the agent moves only if ||F_i|| > a (strict)
      integrate v_i = (dt / m_i) F_i             (overdamped explicit step)
      cap       if ||v_i|| > max_disp: v_i <- v_i * max_disp / ||v_i||
      move      p_i <- p_i + u_i, diameters unchanged.

  Pair search: brute force over all O(n^2) pairs is the definition
  (pairs_bruteforce).  pairs_kdtree finds the same set with scipy's cKDTree as
  a candidate filter followed by the identical FP64 test; tests pin the two
  equal, and large inputs use the kd-tree form.

  Grid (Sec. IV-A, Fig. 4): the box an agent falls in is computed in FP32 on
  purpose, because floating point decides an integer there and the library
  decides it in FP32 too:
      S = max_i diameter_i + 2m (the largest contact distance);
      e = S + 8 ulp(C), C = max(S, largest |coordinate|): rounding the box
          coordinate moves an agent by at most ~3 such ulps, so every contact
          pair stays within adjacent boxes, which is what Sec. IV-A relies on;
      o = min_i p_i - e  (per axis);
      b = max(floor((p - o) / e), 1);  dims = max(floor((max_i p_i - o) / e), 1) + 2;
      key = (b_z * dims_y + b_y) * dims_x + b_x;  boxes listed in key order.
  Within a box the paper fixes no order (Sec. IV-D sorts for locality); the
  library's reading, restated here: the box edge is cut into K = 2^ks slices
  along x, ks the largest of 0..3 with 4 * K * nboxes <= 5 * n, and agents are
  ordered by their slice sx = floor((t_x - b_x) * K) (clamped to [0, K)), with
  t = (p - o) / e the float32 position in box units, then by input index
  (stable).

All floating-point inputs, including parameters, are the float32 values the GPU
sees, widened exactly to float64.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

F32 = np.float32


@dataclass
class Params:
    """Mechanical constants.  kappa, gamma: Eq. 1.  adherence, dt, density,
    max_disp: the Sec. III displacement rules (readings).  contact_margin widens
    delta and the box edge."""
    k: float = 2.0
    gamma: float = 1.0
    adherence: float = 0.1
    dt: float = 1.0
    density: float = 0.02
    max_disp: float = 3.0
    contact_margin: float = 0.0

    def as64(self) -> "Params":
        """The float32-rounded values, widened to float64 (what the GPU sees)."""
        return Params(*[float(F32(getattr(self, f))) for f in
                        ("k", "gamma", "adherence", "dt", "density", "max_disp",
                         "contact_margin")])


# --------------------------------------------------------------------- grid (FP32)
def sub_bin_shift(n_agents: int, nboxes: int) -> int:
    """log2 of the x slices per box: the largest ks in 0..3 with
    4 * 2^ks * nboxes <= 5 * n_agents (0 for an empty grid)."""
    ks = 0
    while nboxes > 0 and ks < 3 and 4 * (nboxes << (ks + 1)) <= 5 * n_agents:
        ks += 1
    return ks


def grid(state32: np.ndarray, contact_margin: float = 0.0) -> dict:
    """Uniform grid of Sec. IV-A, box edge = largest diameter (+2 margin).

    Returns origin, edge, dims, per-agent box coords and key, box counts and the
    exclusive start table (length nboxes + 1), the x slices per box (ks, and
    each agent's slice sx), the table of slice starts (length K nboxes + 1,
    slice sx of box k at entry k K + sx), and the sorting permutation (sorted
    slot -> input index: by box, then slice, then input index)."""
    st = np.ascontiguousarray(state32, dtype=F32)
    p = st[:, :3]
    m2 = F32(2.0) * F32(contact_margin)
    S = F32(st[:, 3].max()) + m2                  # largest contact distance
    lo = p.min(axis=0)
    hi = p.max(axis=0)
    C = max(S, np.abs(lo).max(), np.abs(hi).max())
    e = F32(S + F32(8.0) * (np.nextafter(C, F32(np.inf)) - C))
    o = (lo - e).astype(F32)
    t = ((p - o) / e).astype(F32)                 # position in box units, float32
    b = np.floor(t).astype(np.int64)
    b = np.maximum(b, 1)
    dims = np.maximum(np.floor((hi - o) / e).astype(np.int64), 1) + 2
    key = (b[:, 2] * dims[1] + b[:, 1]) * dims[0] + b[:, 0]
    nboxes = int(dims[0] * dims[1] * dims[2])
    counts = np.bincount(key, minlength=nboxes)
    start = np.zeros(nboxes + 1, dtype=np.int64)
    start[1:] = np.cumsum(counts)
    ks = sub_bin_shift(len(st), nboxes)
    K = 1 << ks
    frac = (t[:, 0] - b[:, 0].astype(F32)).astype(F32)      # exact in float32
    sx = np.clip(np.floor(frac * F32(K)).astype(np.int64), 0, K - 1)
    skey = key * K + sx
    table = np.zeros(K * nboxes + 1, dtype=np.int64)
    table[1:] = np.cumsum(np.bincount(skey, minlength=K * nboxes))
    perm = np.argsort(skey, kind="stable")
    return dict(origin=o, edge=F32(e), dims=dims, box=b, key=key, nboxes=nboxes,
                counts=counts, start=start, ks=ks, sub=sx, table=table, perm=perm)


# --------------------------------------------------------------------- pairs (FP64)
def _contact_test(pi, pj, ri, rj, m):
    diff = pi - pj
    d = np.sqrt(np.sum(diff * diff, axis=-1))
    delta = ri + rj + 2.0 * m - d
    return delta, d


def pairs_bruteforce(pos: np.ndarray, rad: np.ndarray, margin: float = 0.0,
                     chunk: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """All ordered pairs (i, j), i != j, with delta > 0 and d > 0, by testing
    every pair.  Returned sorted by (i, j)."""
    n = len(pos)
    if chunk <= 0:
        chunk = max(1, min(n, 4_000_000 // max(n, 1)))
    I, J = [], []
    for i0 in range(0, n, chunk):
        i1 = min(n, i0 + chunk)
        delta, d = _contact_test(pos[i0:i1, None, :], pos[None, :, :],
                                 rad[i0:i1, None], rad[None, :], margin)
        mask = (delta > 0.0) & (d > 0.0)
        mask[np.arange(i1 - i0), np.arange(i0, i1)] = False
        ii, jj = np.nonzero(mask)
        I.append(ii + i0)
        J.append(jj)
    I = np.concatenate(I) if I else np.zeros(0, np.int64)
    J = np.concatenate(J) if J else np.zeros(0, np.int64)
    return I.astype(np.int64), J.astype(np.int64)


def pairs_kdtree(pos: np.ndarray, rad: np.ndarray, margin: float = 0.0
                 ) -> tuple[np.ndarray, np.ndarray]:
    """Same set as pairs_bruteforce: cKDTree proposes every pair closer than the
    largest possible contact distance, then the identical FP64 test decides."""
    from scipy.spatial import cKDTree

    n = len(pos)
    if n < 2:
        z = np.zeros(0, np.int64)
        return z, z
    rmax = 2.0 * float(rad.max()) + 2.0 * margin
    cand = cKDTree(pos).query_pairs(r=rmax * (1.0 + 1e-9) + 1e-12, output_type="ndarray")
    if len(cand) == 0:
        z = np.zeros(0, np.int64)
        return z, z
    a, b = cand[:, 0].astype(np.int64), cand[:, 1].astype(np.int64)
    delta, d = _contact_test(pos[a], pos[b], rad[a], rad[b], margin)
    keep = (delta > 0.0) & (d > 0.0)
    a, b = a[keep], b[keep]
    I = np.concatenate([a, b])
    J = np.concatenate([b, a])
    order = np.lexsort((J, I))
    return I[order], J[order]


def find_pairs(pos, rad, margin=0.0, method="auto"):
    if method == "auto":
        method = "brute" if len(pos) <= 1500 else "kdtree"
    if method == "brute":
        return pairs_bruteforce(pos, rad, margin)
    return pairs_kdtree(pos, rad, margin)


# --------------------------------------------------------------------- forces (Eq. 1)
def pair_terms(pos, diam, prm: Params, I, J):
    """Per ordered pair: delta, d, R, phi, unit vector u = (p_i - p_j)/d."""
    m = prm.contact_margin
    r = 0.5 * diam
    diff = pos[I] - pos[J]
    d = np.sqrt(np.sum(diff * diff, axis=1))
    delta = r[I] + r[J] + 2.0 * m - d
    R = r[I] * r[J] / (r[I] + r[J])
    root = np.sqrt(R * delta)
    phi = prm.k * delta - prm.gamma * root
    u = diff / d[:, None]
    return dict(delta=delta, d=d, R=R, root=root, phi=phi, u=u)


def forces(pos, diam, prm: Params, I, J):
    """F_i = sum_j f_ij (Eq. 1) plus the condition scale
    S_i = sum_j (kappa delta_ij + gamma sqrt(R_ij delta_ij)) and pair counts."""
    n = len(pos)
    t = pair_terms(pos, diam, prm, I, J)
    f = t["phi"][:, None] * t["u"]
    F = np.stack([np.bincount(I, weights=f[:, c], minlength=n) for c in range(3)], axis=1)
    S = np.bincount(I, weights=prm.k * t["delta"] + prm.gamma * t["root"], minlength=n)
    npairs = np.bincount(I, minlength=n)
    return F, S, npairs, t


# --------------------------------------------------------------------- displacement
def mass(diam, prm: Params):
    return prm.density * (np.pi / 6.0) * diam ** 3


def displacement(F, diam, prm: Params):
    """Adherence test, integration and cap of Sec. III (readings in the module
    docstring).  Returns u, v (uncapped), moving and capped flags."""
    Fn = np.linalg.norm(F, axis=1)
    moving = Fn > prm.adherence
    m = mass(diam, prm)
    v = (prm.dt / m)[:, None] * F
    vn = np.linalg.norm(v, axis=1)
    capped = moving & (vn > prm.max_disp)
    u = np.where(moving[:, None], v, 0.0)
    if capped.any():
        u[capped] = v[capped] * (prm.max_disp / vn[capped])[:, None]
    return dict(u=u, v=v, Fn=Fn, vn=vn, moving=moving, capped=capped)


# --------------------------------------------------------------------- one step
def step(state, prm: Params = Params(), method="auto", pairs=None):
    """One mechanical-interaction step.  `state` is (n, 4) rows (x, y, z, d) in
    float32 or float64; float32 input is widened exactly."""
    prm64 = prm.as64()
    st = np.asarray(state, dtype=np.float64)
    pos, diam = st[:, :3], st[:, 3]
    if pairs is None:
        pairs = find_pairs(pos, 0.5 * diam, prm64.contact_margin, method)
    I, J = pairs
    F, S, npairs, terms = forces(pos, diam, prm64, I, J)
    disp = displacement(F, diam, prm64)
    new = st.copy()
    new[:, :3] += disp["u"]
    return dict(state=new, F=F, S=S, npairs=npairs, I=I, J=J, terms=terms, **disp)


def trajectory(state0, prm: Params = Params(), nsteps: int = 1, method="auto",
               keep=False):
    """Iterate `step`; positions stay float64 throughout.  With keep=True every
    step's record is returned as well."""
    st = np.asarray(state0, dtype=np.float64).copy()
    recs = []
    for _ in range(nsteps):
        r = step(st, prm, method)
        if keep:
            recs.append(dict(state=st, **{k: v for k, v in r.items() if k != "state"}))
        st = r["state"]
    return (st, recs) if keep else st


# --------------------------------------------------------------------- sampled form
def step_sampled(state, idx, prm: Params = Params()):
    """The step's F, S, contact count and displacement for the rows in `idx`
    only, each against every row (agent by agent, for populations too large
    for `step`).  Candidates come from a cKDTree ball query, the contact test
    and Eq. 1 are the same FP64 expressions as in `pair_terms`."""
    from scipy.spatial import cKDTree

    prm64 = prm.as64()
    st = np.asarray(state, dtype=np.float64)
    pos, diam = st[:, :3], st[:, 3]
    rad = 0.5 * diam
    idx = np.asarray(idx, dtype=np.int64)
    rmax = 2.0 * float(rad.max()) + 2.0 * prm64.contact_margin
    lists = cKDTree(pos).query_ball_point(pos[idx], r=rmax * (1.0 + 1e-9) + 1e-12)
    I = np.concatenate([np.full(len(l), k, np.int64) for k, l in enumerate(lists)]) if len(idx) else np.zeros(0, np.int64)
    J = np.concatenate([np.asarray(l, np.int64) for l in lists]) if len(idx) else np.zeros(0, np.int64)
    gi = idx[I]
    keep = gi != J
    gi, J, I = gi[keep], J[keep], I[keep]
    delta, d = _contact_test(pos[gi], pos[J], rad[gi], rad[J], prm64.contact_margin)
    keep = (delta > 0.0) & (d > 0.0)
    gi, J, I = gi[keep], J[keep], I[keep]
    t = pair_terms(pos, diam, prm64, gi, J)
    f = t["phi"][:, None] * t["u"]
    m = len(idx)
    F = np.stack([np.bincount(I, weights=f[:, c], minlength=m) for c in range(3)], axis=1)
    S = np.bincount(I, weights=prm64.k * t["delta"] + prm64.gamma * t["root"], minlength=m)
    npairs = np.bincount(I, minlength=m)
    disp = displacement(F, diam[idx], prm64)
    return dict(F=F, S=S, npairs=npairs, I=idx[I], J=J, delta=t["delta"], **disp)


# --------------------------------------------------------------------- adjoint
def mse_loss(pos, target):
    diff = pos - target
    return float(np.sum(diff * diff) / diff.size)


def trajectory_grad(state0, target_pos, prm: Params = Params(), nsteps: int = 1,
                    method="auto"):
    """Loss L = mean over coordinates of (p_T - target)^2 after nsteps, and its
    gradient with respect to kappa, gamma, the initial positions and diameters.

    Reverse pass (chain rule through the step above; the adherence indicator,
    the cap branch and pair membership are piecewise constant):
      w_i = dL/du_i = dL/dp_i(t+1)
      capped:  w_i <- (max_disp/|v_i|) (I - v^ v^T) w_i
      g_i = (dt/m_i) w_i if moving else 0                       (= dL/dF_i)
      dL/dm_i = -(w_i . v_i)/m_i if moving
      J_ij = phi'(d) u u^T + (phi/d)(I - u u^T),  phi'(d) = -(kappa - gamma R/(2 sqrt(R delta)))
      dL/dp_i(t) = dL/dp_i(t+1) + sum_j J_ij (g_i - g_j)
      dL/dkappa += sum_(i,j) g_i . delta_ij u_ij
      dL/dgamma -= sum_(i,j) g_i . sqrt(R_ij delta_ij) u_ij
      dL/dd_i(t) = dL/dd_i(t+1) + dL/dm_i * 3 m_i / d_i
                   + sum_j (g_i - g_j) . u_ij * (1/2) dphi/dr_i,
        dphi/dr_i = (kappa - gamma R/(2 sqrt(R delta))) - gamma delta/(2 sqrt(R delta)) * r_j^2/(r_i+r_j)^2
    """
    final, recs = trajectory(state0, prm, nsteps, method, keep=True)
    return _reverse(recs, final, target_pos, prm)


def trajectory_grad_along(states, target_pos, prm: Params = Params(), method="auto"):
    """The reverse pass of `trajectory_grad` along given forward states
    X_0 .. X_T (for instance another implementation's float32 rows, in id
    order): each step is linearised at the given X_t by evaluating `step` there,
    and the loss is taken on the given X_T."""
    recs = []
    for X in states[:-1]:
        X = np.asarray(X, dtype=np.float64)
        r = step(X, prm, method)
        recs.append(dict(state=X, **{k: v for k, v in r.items() if k != "state"}))
    return _reverse(recs, np.asarray(states[-1], dtype=np.float64), target_pos, prm)


def _reverse(recs, final, target_pos, prm: Params):
    prm64 = prm.as64()
    tgt = np.asarray(target_pos, dtype=np.float64)
    n = final.shape[0]
    L = mse_loss(final[:, :3], tgt)
    Gp = 2.0 * (final[:, :3] - tgt) / (3.0 * n)
    Gd = np.zeros(n)
    dk = 0.0
    dg = 0.0
    for rec in reversed(recs):
        st = rec["state"]
        diam = st[:, 3]
        rad = 0.5 * diam
        I, J, t = rec["I"], rec["J"], rec["terms"]
        w = Gp.copy()
        moving, capped, v, vn = rec["moving"], rec["capped"], rec["v"], rec["vn"]
        if capped.any():
            vh = v[capped] / vn[capped][:, None]
            wc = w[capped]
            w[capped] = (prm64.max_disp / vn[capped])[:, None] * (
                wc - vh * np.sum(vh * wc, axis=1)[:, None])
        m = mass(diam, prm64)
        g = np.where(moving[:, None], (prm64.dt / m)[:, None] * w, 0.0)
        dLdm = np.where(moving, -np.sum(w * v, axis=1) / m, 0.0)
        # pair Jacobian applied to (g_i - g_j)
        u, d, delta, R, root, phi = t["u"], t["d"], t["delta"], t["R"], t["root"], t["phi"]
        dphi_ddelta = prm64.k - prm64.gamma * R / (2.0 * root)
        dphi_dd = -dphi_ddelta
        gd = g[I] - g[J]
        ug = np.sum(u * gd, axis=1)
        Jg = dphi_dd[:, None] * u * ug[:, None] + (phi / d)[:, None] * (gd - u * ug[:, None])
        newGp = Gp.copy()
        for c in range(3):
            newGp[:, c] += np.bincount(I, weights=Jg[:, c], minlength=n)
        gi_u = np.sum(g[I] * u, axis=1)
        dk += float(np.sum(gi_u * delta))
        dg -= float(np.sum(gi_u * root))
        ri, rj = rad[I], rad[J]
        dphi_dR = -prm64.gamma * delta / (2.0 * root)
        dphi_dri = dphi_ddelta + dphi_dR * rj * rj / ((ri + rj) ** 2)
        newGd = Gd + dLdm * 3.0 * m / diam
        newGd += np.bincount(I, weights=ug * 0.5 * dphi_dri, minlength=n)
        Gp, Gd = newGp, newGd
    return dict(loss=L, dk=dk, dgamma=dg, dpos=Gp, ddiam=Gd, final=final)


def trajectory_loss(state0, target_pos, prm: Params = Params(), nsteps: int = 1,
                    method="auto") -> float:
    final = trajectory(state0, prm, nsteps, method)
    return mse_loss(final[:, :3], np.asarray(target_pos, dtype=np.float64))


# --------------------------------------------------------------------- diagnostics
def margins(rec, prm: Params = Params()):
    """How close a step came to a piecewise boundary: smallest |F|-a relative to
    S, smallest |v|-max_disp, smallest delta.  Used to pick FD-safe fixtures and to
    flag adherence flips when comparing with a float32 result."""
    prm64 = prm.as64()
    S = np.maximum(rec["S"], 1e-300)
    adh = np.abs(rec["Fn"] - prm64.adherence) / S
    cap = np.abs(rec["vn"][rec["moving"]] - prm64.max_disp) if rec["moving"].any() else np.array([np.inf])
    dmin = rec["terms"]["delta"].min() if len(rec["I"]) else np.inf
    return dict(adherence=adh, cap=cap, min_delta=dmin)
