"""torch.autograd wrapper of qsim_rollout_vjp (differentiable H-step quadrotor rollout).

The forward pass and the reverse sweep both run in libqsim; this module only allocates the
workspace with torch and routes ``grad_output`` into the library as the per-env seed.
"""
from __future__ import annotations

import torch

from . import (QsimParams, QsimVjpDesc, _lib, load, qsim_rollout_vjp, qsim_vjp_workspace)


def make_desc(n, ld, H, ckpt, mode, weights, dt=0.01, renorm=1, n_hist=16, hidden=64,
              lanes_per_env=0):
    d = QsimVjpDesc()
    d.n, d.ld, d.H, d.ckpt, d.mode = int(n), int(ld), int(H), int(ckpt), int(mode)
    d.n_hist, d.hidden = int(n_hist), int(hidden)
    d.lanes_per_env = int(lanes_per_env)
    d.w_p, d.w_q, d.w_v, d.w_a = (float(x) for x in weights)
    d.dt, d.renorm = float(dt), int(renorm)
    return d


def _workspace(desc):
    nbytes = qsim_vjp_workspace(desc)
    return torch.empty((nbytes + 3) // 4, dtype=torch.float32, device="cuda")


class RolloutLoss(torch.autograd.Function):
    """loss_e of an H-step rollout; differentiable w.r.t. ``params`` rows m, Jx, Jy, Jz
    and w.r.t. ``x`` = actions [H][4][ld] (open loop) or the flat actor (closed loop)."""

    @staticmethod
    def forward(ctx, params, x, s0, veh: QsimParams, desc: QsimVjpDesc):
        load()
        ld, n = desc.ld, desc.n
        loss = torch.zeros(ld, device="cuda")
        ws = _workspace(desc)
        acts = x if desc.mode == 0 else None
        actor = x if desc.mode == 1 else None
        qsim_rollout_vjp(desc, veh, s0, params, acts, actor, None, loss, None, None, None, None,
                         ws)
        ctx.save_for_backward(params, x, s0)
        ctx.veh, ctx.desc = veh, desc
        return loss[:n]

    @staticmethod
    def backward(ctx, g_loss):
        params, x, s0 = ctx.saved_tensors
        desc, veh = ctx.desc, ctx.veh
        ld, n = desc.ld, desc.n
        seed = torch.zeros(ld, device="cuda")
        seed[:n] = g_loss
        loss = torch.zeros(ld, device="cuda")
        gp = torch.zeros(4, ld, device="cuda")
        ws = _workspace(desc)
        if desc.mode == 0:
            gx = torch.zeros_like(x)
            qsim_rollout_vjp(desc, veh, s0, params, x, None, seed, loss, gx, None, gp, None, ws)
        else:
            gx = torch.zeros_like(x)
            qsim_rollout_vjp(desc, veh, s0, params, None, x, seed, loss, None, gx, gp, None, ws)
        g_params = torch.zeros_like(params)
        g_params[0:4] = gp
        return g_params, gx, None, None, None


def rollout_loss(s0, params, veh, H, ckpt, weights, actions=None, actor=None, n_hist=16,
                 hidden=64, dt=0.01, renorm=1):
    """Per-env loss of an H-step rollout from states ``s0`` [17][ld] with per-env
    ``params`` [8][ld]; pass ``actions`` [H][4][ld] (open loop) or a flat ``actor``."""
    ld = s0.shape[1]
    n = ld if not hasattr(s0, "n_envs") else s0.n_envs
    mode = 0 if actions is not None else 1
    desc = make_desc(n, ld, H, ckpt, mode, weights, dt, renorm, n_hist, hidden)
    return RolloutLoss.apply(params, actions if mode == 0 else actor, s0, veh, desc)
