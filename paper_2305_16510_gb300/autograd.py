"""torch.autograd.Function over the differentiable rollout of the C-ABI.

forward: ag_set_state / ag_set_gains, then ag_rollout_loss (recorded forward
in libaerialgb); backward: ag_backward (the hand-written adjoint kernel).
Torch only carries the tensors; every derivative is computed by the library.
"""
from __future__ import annotations

import torch

from . import _abi


class RolloutLoss(torch.autograd.Function):
    """loss[i] = sum_t w_pos |p_t - p_goal_i|^2 + w_omega |Omega_t|^2 over n_steps steps.

    Inputs: x0 float32 [13, n] (initial state), gains float32 [12] and,
    optionally, targets float32 [4, n] (each environment's command targets,
    differentiable too; None keeps the fleet's commands); the fleet, its
    initial motors [8, n], the horizon, the goals [3, n] and the weights are
    constants. Returns float32 [n] on the fleet's device.

    The library keeps one recorded rollout per fleet: a second forward on the
    same fleet replaces the first one's tape, and the first one's backward
    then raises instead of returning the gradients of the other rollout.
    """

    @staticmethod
    def forward(ctx, x0, gains, targets, fleet, motors0, n_steps, p_goal, w_pos, w_omega):
        if targets is not None:
            fleet.set_commands(None, targets.detach())
        fleet.set_state(x0.detach(), motors0)
        _abi.ag_set_gains(fleet.ctx, gains.detach().to("cpu", torch.float32).contiguous())
        loss = torch.empty(fleet.n, dtype=torch.float32, device=fleet.device)
        goal = p_goal.to(device=fleet.device, dtype=torch.float32).contiguous()
        _abi.ag_rollout_loss(fleet.ctx, n_steps, w_pos, w_omega, goal, loss)
        fleet._recording = getattr(fleet, "_recording", 0) + 1
        ctx.recording = fleet._recording
        ctx.fleet = fleet
        ctx.gains_device = gains.device
        ctx.has_targets = targets is not None
        ctx._keep = goal
        return loss

    @staticmethod
    def backward(ctx, grad_loss):
        fleet = ctx.fleet
        if getattr(fleet, "_recording", 0) != ctx.recording:
            raise RuntimeError("the fleet recorded another rollout after this loss was computed: its backward "
                               "would differentiate that rollout instead")
        gx = torch.empty((13, fleet.n), dtype=torch.float32, device=fleet.device)
        gg = torch.empty((12,), dtype=torch.float32, device=fleet.device)
        gt = torch.empty((4, fleet.n), dtype=torch.float32, device=fleet.device) if ctx.has_targets else None
        w = grad_loss.to(device=fleet.device, dtype=torch.float32).contiguous()
        _abi.ag_backward(fleet.ctx, w, gx, gg, None, gt)
        return gx, gg.to(ctx.gains_device), gt, None, None, None, None, None, None


def rollout_loss(fleet, x0, gains, motors0, n_steps: int, p_goal, w_pos: float = 1.0, w_omega: float = 0.01,
                 targets=None):
    """Differentiable per-environment rollout loss (see RolloutLoss)."""
    return RolloutLoss.apply(x0, gains, targets, fleet, motors0, int(n_steps), p_goal, float(w_pos), float(w_omega))
