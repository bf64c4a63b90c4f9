"""Gym-style vectorised environment for the reach-a-setpoint task.

The paper trains policies that fly multirotors to a goal setpoint through the
attitude or velocity command interface (Sec. I). ``ReachEnv`` exposes that
task over a fleet in the reset/step form RL code expects, with every
environment on the GPU and no per-step host synchronisation: actions, the
fleet step, rewards, terminations, auto-resets and observations all run in
libaerialgb's kernels (ag_reach_step). Tensors are torch tensors on the
fleet's device, batch-major: actions [n, 4], observations [n, 13].
"""
from __future__ import annotations

import torch

from . import _abi
from .fleet import Fleet

OBS_DIM = 13
ACTION_DIM = 4


class ReachEnv:
    """Reach-a-setpoint over n_envs vehicles.

    ``reset()`` draws fresh episodes (ag_reset) and returns the first
    observations; ``step(actions)`` returns (obs, reward, done, info) where an
    environment whose episode ended has already been reset and ``obs`` shows
    its new episode. ``info["collided"]`` marks the episodes that ended in a
    collision. Actions lie in [-1, 1] (clamped) and map to commands through
    ``task.action_scale`` and ``task.action_offset``. The returned tensors are
    the environment's own buffers, overwritten by the next step (so that a
    step allocates nothing): clone what must outlive it.
    """

    def __init__(self, n_envs: int, goals=None, task: _abi.ag_reach_config | None = None, seed: int = 1,
                 **fleet_kwargs):
        self.fleet = Fleet(n_envs, seed=seed, **fleet_kwargs)
        self.n = n_envs
        self.seed = seed
        self.task = _abi.ag_reach_config_default() if task is None else task
        dev = self.fleet.device
        self.goals = (torch.zeros((3, n_envs), dtype=torch.float32, device=dev) if goals is None
                      else torch.as_tensor(goals, dtype=torch.float32).to(dev).contiguous())
        if tuple(self.goals.shape) != (3, n_envs):
            raise ValueError("goals must have shape (3, n_envs)")
        self.obs = torch.empty((n_envs, OBS_DIM), dtype=torch.float32, device=dev)
        self.reward = torch.empty((n_envs,), dtype=torch.float32, device=dev)
        self.done = torch.empty((n_envs,), dtype=torch.uint8, device=dev)
        self._col = torch.empty((n_envs,), dtype=torch.uint8, device=dev)

    @property
    def device(self) -> torch.device:
        return self.fleet.device

    def reset(self, seed: int | None = None) -> torch.Tensor:
        if seed is not None:
            self.seed = seed
        self.fleet.reset(None, self.seed)
        _abi.ag_reach_begin(self.fleet.ctx, self.task, self.goals)
        _abi.ag_reach_observe(self.fleet.ctx, self.obs)
        return self.obs

    def step(self, actions: torch.Tensor):
        a = actions
        if a.dtype != torch.float32 or a.device != self.device or not a.is_contiguous() or a.data_ptr() % 16:
            a = a.to(device=self.device, dtype=torch.float32).contiguous().clone()
        if tuple(a.shape) != (self.n, ACTION_DIM):
            raise ValueError(f"actions must have shape ({self.n}, {ACTION_DIM})")
        _abi.ag_reach_step(self.fleet.ctx, a, self.obs, self.reward, self.done)
        _abi.ag_get_state(self.fleet.ctx, collided=self._col)
        self._keep_actions = a
        return self.obs, self.reward, self.done, {"collided": self._col}

    def close(self) -> None:
        self.fleet.close()
