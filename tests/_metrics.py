"""Error metrics for comparing the float32 CUDA path with the FP64 oracle.

Per agent, a force error is measured against the agent's condition scale
S_i = sum_j (kappa delta_ij + gamma sqrt(R_ij delta_ij)) (the sum of the
magnitudes of its pair terms) or |F_i| if larger: a relative error of the sum
itself is ill-conditioned when the pair forces cancel.  Displacements use the
same scale times dt/m_i.  Agents with no contact must get exactly zero.
"""
import math

import numpy as np

TOL_STEP = 1e-5        # per-step tolerance on forces and displacements
TOL_TRAJ = 1e-3        # tolerance after many steps


def by_id(rows_sorted: np.ndarray, perm: np.ndarray) -> np.ndarray:
    out = np.empty_like(rows_sorted)
    out[perm] = rows_sorted
    return out


def force_errors(Fg, F, S):
    """(max per-agent error, norm-wise error, number of contact-free agents with
    a nonzero GPU force)."""
    Fg = np.asarray(Fg, dtype=np.float64)
    scale = np.maximum(np.linalg.norm(F, axis=1), S)
    diff = np.linalg.norm(Fg - F, axis=1)
    zero = scale == 0
    bad_zero = int(np.count_nonzero(diff[zero]))
    per = diff[~zero] / scale[~zero] if (~zero).any() else np.zeros(1)
    norm = float(np.linalg.norm(Fg - F) / max(np.linalg.norm(F), 1e-300))
    return float(per.max()), norm, bad_zero


def mass(diam, density=0.02):
    return float(np.float32(density)) * (math.pi / 6.0) * np.asarray(diam, np.float64) ** 3


def adherence_flips(Fn_ref, S, adherence):
    """Agents whose |F| lies within the per-step tolerance of the adherence
    threshold: float32 and float64 may legitimately decide them differently."""
    a = float(np.float32(adherence))
    return np.abs(Fn_ref - a) <= TOL_STEP * np.maximum(S, 1e-300)


def disp_errors(ug, u, S, diam, dt=1.0, density=0.02, exclude=None):
    ug = np.asarray(ug, dtype=np.float64)
    scale = np.maximum(np.linalg.norm(u, axis=1), S * float(np.float32(dt)) / mass(diam, density))
    diff = np.linalg.norm(ug - u, axis=1)
    keep = np.ones(len(u), bool) if exclude is None else ~exclude
    zero = (scale == 0) & keep
    bad_zero = int(np.count_nonzero(diff[zero]))
    sel = keep & (scale > 0)
    per = diff[sel] / scale[sel] if sel.any() else np.zeros(1)
    return float(per.max()), bad_zero


def ulp32(x):
    x = np.abs(np.asarray(x, np.float32))
    return (np.nextafter(x, np.float32(np.inf)) - x).astype(np.float64)


def record(quantity: str, **values):
    """Append one measured error to the JSON-lines file named by the
    PARITY_REPORT environment variable (nothing happens when it is unset): the
    per-quantity error table is assembled from these records."""
    import json
    import os
    path = os.environ.get("PARITY_REPORT")
    if not path:
        return
    row = {"quantity": quantity}
    row.update({k: (float(v) if isinstance(v, (np.floating, np.integer)) else v) for k, v in values.items()})
    with open(path, "a") as f:
        f.write(json.dumps(row) + "\n")
