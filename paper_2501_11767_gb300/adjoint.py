"""Gradients of a final-morphology functional through many steps.

Orchestration only: every step, every adjoint step and the functional run
in the CUDA library (chnss_step, chnss_adjoint_step, chnss_objective).

trajectory_gradient() runs `steps` forward steps keeping a checkpoint every
`checkpoint_every` steps (device copies), then walks the segments backwards:
each segment is recomputed from its checkpoint and traversed with
chnss_adjoint_step.  Memory: (steps / k + k) states instead of steps + 1.

FilmGradient is a torch.autograd.Function of (phi_p0, evap_rate, gamma)
returning J = int |grad phi_p(t_m)|^2; its backward uses the same sweep.
"""
from __future__ import annotations

import torch

from . import chnss


def _clone(state):
    return {k: v.clone() for k, v in state.items()}


def trajectory_gradient(ctx: "chnss.Context", state0: dict, steps: int, checkpoint_every: int = 8):
    """J(t_m) and its gradient: dict(evap=, gamma=, adj0= adjoint state at
    t_0 (adj0["phi"][0] is dJ/dphi_p0), J=)."""
    k = max(1, checkpoint_every)
    ckpt = {0: _clone(state0)}
    cur = _clone(state0)
    for i in range(steps):
        nxt, _, _ = ctx.step(cur)
        cur = nxt
        if (i + 1) % k == 0 and (i + 1) < steps:
            ckpt[i + 1] = _clone(cur)
    final = cur
    lam = ctx.new_state()
    J = ctx.objective(final["phi"][0], lam["phi"][0])
    grad = [0.0, 0.0]
    end = steps
    for start in sorted(ckpt, reverse=True):
        seg = [ckpt[start]]
        for _ in range(start, end):
            nxt, _, _ = ctx.step(seg[-1])
            seg.append(nxt)
        for j in range(end - start, 0, -1):
            lam, g, _, _ = ctx.adjoint_step(seg[j - 1], seg[j], lam)
            grad[0] += g[0]
            grad[1] += g[1]
        end = start
    return {"J": J, "evap": grad[0], "gamma": grad[1], "adj0": lam}


class FilmGradient(torch.autograd.Function):
    """J = int |grad phi_p(t_m)|^2 as a differentiable function of the initial
    polymer field, the evaporation rate and the mobility scale."""

    @staticmethod
    def forward(fctx, phi_p0, evap_rate, gamma, mesh, params, state0, steps, checkpoint_every):
        p = dict(params, evap_rate=float(evap_rate), gamma=[float(gamma)] * 3)
        ctx = chnss.Context(mesh, p)
        st = _clone(state0)
        st["phi"][0].copy_(phi_p0)
        out = trajectory_gradient(ctx, st, steps, checkpoint_every)
        fctx.save_for_backward(out["adj0"]["phi"][0].clone())
        fctx.grads = (out["evap"], out["gamma"])
        return torch.tensor(out["J"], dtype=torch.float64)

    @staticmethod
    def backward(fctx, gJ):
        (gphi,) = fctx.saved_tensors
        ge, gg = fctx.grads
        s = float(gJ)
        return (gphi * s, torch.tensor(ge * s, dtype=torch.float64), torch.tensor(gg * s, dtype=torch.float64),
                None, None, None, None, None)
