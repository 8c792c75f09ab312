"""Differentiable ORCA rollouts for PyTorch.

``rollout(sim, pos0, vel0, goal, radius, max_speed, pref_speed, time_horizon, T)`` returns
the positions p(1..T) (CUDA tensor [T, n, 2]) of T synchronous ORCA steps computed by the
library, as a differentiable function of pos0, vel0, radius, pref_speed and time_horizon.
The backward pass is the library's hand-written adjoint (orca_rollout_backward): each step
is differentiated through the constraints that fixed the selected velocity, with the
neighbour sets and all branches held fixed, re-running each checkpoint segment
(``ckpt_every`` steps) to recover the records it needs, or, with ``ckpt_every = 0``,
sweeping the records the forward pass kept of every step ((20 + 4 k) bytes per
agent-step of device memory, no recomputation).  goal and max_speed get no gradient.

Any loss built from the trajectory in PyTorch can then be back-propagated, e.g. the mean
squared position error against a target rollout.
"""
from __future__ import annotations

import torch

from . import abi


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos0, vel0, goal, radius, max_speed, pref_speed, time_horizon, sim, T,
                ckpt_every):
        n = pos0.shape[0]
        args = [t.detach().contiguous().float() for t in
                (pos0, vel0, goal, radius, max_speed, pref_speed, time_horizon)]
        sim.set_agents(*args)
        nbytes = abi.orca_rollout_workspace_size(sim.ctx, T, ckpt_every)
        raw = torch.empty(nbytes + 256, dtype=torch.uint8, device=pos0.device)
        off = (-raw.data_ptr()) % 256
        ws = raw[off: off + nbytes]
        traj = torch.empty((T, n, 2), dtype=torch.float32, device=pos0.device)
        abi.orca_rollout_forward(sim.ctx, T, ckpt_every, traj, ws)
        ctx.sim, ctx.ws, ctx.raw, ctx.n = sim, ws, raw, n
        return traj

    @staticmethod
    def backward(ctx, g_traj):
        n, dev = ctx.n, g_traj.device
        g = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(3)]
        gp0 = torch.empty((n, 2), dtype=torch.float32, device=dev)
        gv0 = torch.empty((n, 2), dtype=torch.float32, device=dev)
        abi.orca_rollout_backward(ctx.sim.ctx, g_traj.contiguous().float(), g[0], g[1], g[2], gp0,
                                  gv0, ctx.ws)
        # order of forward's inputs: pos0, vel0, goal, radius, max_speed, pref_speed, tau, ...
        return gp0, gv0, None, g[1], None, g[0], g[2], None, None, None


def rollout(sim, pos0, vel0, goal, radius, max_speed, pref_speed, time_horizon, T: int,
            ckpt_every: int = 8):
    """Positions p(1..T) [T, n, 2] of a rollout from (pos0, vel0); differentiable."""
    return _Rollout.apply(pos0, vel0, goal, radius, max_speed, pref_speed, time_horizon, sim,
                          int(T), int(ckpt_every))


def mse_trajectory_loss(traj, target):
    """(1/(T n)) sum_t sum_i |p_i(t) - target_i(t)|^2."""
    T, n = traj.shape[0], traj.shape[1]
    return ((traj - target) ** 2).sum() / (T * n)
