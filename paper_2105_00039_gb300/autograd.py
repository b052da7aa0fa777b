"""Differentiable trajectories: torch.autograd.Function over the fused step.

Forward runs `nsteps` library steps, keeping a checkpoint of the rows every
`ckpt_every` steps.  Backward calls the library's adjoint (ug_step_backward)
segment by segment in reverse: each segment is recomputed from its checkpoint
with its grids saved, then swept backwards.  Gradients flow to the initial rows
(positions and diameters) and to Eq. 1's kappa and gamma.
"""
from __future__ import annotations

from dataclasses import replace

import torch

from . import ugmech as U


class Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, state0, k, gamma, params: U.Params, nsteps: int, ckpt_every: int,
                max_boxes: int):
        p = replace(params, k=float(k), gamma=float(gamma))
        n = state0.shape[0]
        dev = state0.device
        st = state0.detach().contiguous().clone()
        perm = U.iota(n, dev)
        sp = U.Stepper(n, max_boxes, dev)
        ckpts = []
        done = 0
        while done < nsteps:
            seg = min(ckpt_every, nsteps - done)
            ckpts.append((st.clone(), seg))
            sp.step(st, perm, p, seg)
            done += seg
        sp.check("Trajectory.forward")
        ctx.ckpts = ckpts
        ctx.perm = perm
        ctx.p = p
        ctx.max_boxes = max_boxes
        return U.scatter_rows(st, perm)

    @staticmethod
    def backward(ctx, grad_by_id):
        G = U.gather_rows(grad_by_id.contiguous().float(), ctx.perm)
        n = G.shape[0]
        seg_max = max((s for _, s in ctx.ckpts), default=1)
        ws = U.workspace(U.backward_workspace_bytes(n, ctx.max_boxes, seg_max), G.device)
        dk = torch.zeros((), dtype=torch.float64, device=G.device)
        dg = torch.zeros((), dtype=torch.float64, device=G.device)
        status = U.new_status(G.device)
        for st, seg in reversed(ctx.ckpts):
            G, gp, _ = U.step_backward(st, ctx.p, seg, ctx.max_boxes, G, ws=ws, status=status)
            dk = dk + gp[0].double()
            dg = dg + gp[1].double()
        U.check_status(status, "Trajectory.backward")
        return G, dk.float(), dg.float(), None, None, None, None


def trajectory(state0, k, gamma, params: U.Params = U.Params(), nsteps: int = 1,
               ckpt_every: int = 10, max_boxes: int | None = None):
    """Rows (by id) after nsteps steps, differentiable in state0, k and gamma."""
    if max_boxes is None:
        max_boxes = U.estimate_max_boxes(state0.detach(), params.contact_margin, slack=2.0)
    k = k if torch.is_tensor(k) else torch.tensor(float(k))
    gamma = gamma if torch.is_tensor(gamma) else torch.tensor(float(gamma))
    return Trajectory.apply(state0, k, gamma, params, int(nsteps), int(ckpt_every), int(max_boxes))
