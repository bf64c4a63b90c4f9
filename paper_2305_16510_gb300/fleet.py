"""Python convenience layer over the C-ABI: a fleet context with torch buffers.

PyTorch provides device memory and the current CUDA stream; every
computation happens inside libaerialgb's kernels (see ``_abi``).
"""
from __future__ import annotations

import torch

from . import _abi


class Fleet:
    """One ag_ctx. Arrays are structure-of-arrays over environments.

    Every call runs on the context's stream: torch's current stream when the
    fleet is created, unless ``stream`` is given. Inputs that need a dtype or
    device conversion are converted by torch on its current stream, and the
    tensors the getters return are read back by torch on it too; with a
    ``stream`` of its own, use the fleet under ``torch.cuda.stream(fleet.stream)``
    so that both orders agree.
    """

    def __init__(self, n_envs: int, *, substeps_per_step: int = 1, integrator: int = _abi.AG_INTEG_SIE,
                 n_obstacles: int = 0, n_hexa: int = 0, n_octo: int = 0, dt: float = 0.01,
                 motor_tau: float = 0.03, drag: float = 0.0, sphere_r: float = 0.2, u_max: float = 5.0,
                 arm: float = 0.13, k_yaw: float = 0.016, mass: float = 0.75,
                 inertia=(0.007, 0.007, 0.012), kx=(2, 2, 3), kv=(2, 2, 2), kR=(1.2, 1.2, 0.6),
                 kW=(0.2, 0.2, 0.1), seed: int = 1, hbm_budget_bytes: int = 0, device=None, stream=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        c = _abi.ag_config_default()
        c.n_envs = n_envs
        c.substeps_per_step = substeps_per_step
        c.integrator = integrator
        c.n_obstacles = n_obstacles
        c.n_hexa, c.n_octo = n_hexa, n_octo
        c.n_quad = n_envs - n_hexa - n_octo
        c.dt, c.motor_tau, c.drag, c.sphere_r, c.u_max = dt, motor_tau, drag, sphere_r, u_max
        c.arm, c.k_yaw, c.mass = arm, k_yaw, mass
        c.inertia[:] = list(inertia)
        c.kx[:], c.kv[:], c.kR[:], c.kW[:] = list(kx), list(kv), list(kR), list(kW)
        c.seed = seed
        c.hbm_budget_bytes = hbm_budget_bytes
        self.cfg = c
        self.n = n_envs
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.ctx = _abi.ag_create(c, self.stream.cuda_stream)

    # ------------------------------------------------------------ lifetime --
    def close(self) -> None:
        if getattr(self, "ctx", None):
            _abi.ag_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -------------------------------------------------------------- inputs --
    def _dev(self, x, dtype):
        t = torch.as_tensor(x)
        return t.to(device=self.device, dtype=dtype).contiguous()

    def set_commands(self, modes=None, targets=None) -> None:
        m = None if modes is None else self._dev(modes, torch.uint8)
        t = None if targets is None else self._dev(targets, torch.float32)
        _abi.ag_set_commands(self.ctx, m, t)
        self._keep = (m, t)  # the copies are stream-ordered: keep sources alive until the next sync

    def set_obstacles(self, boxes) -> None:
        b = self._dev(boxes, torch.float32)
        _abi.ag_set_obstacles(self.ctx, b)
        self._keep_boxes = b

    def obstacles(self) -> torch.Tensor:
        out = torch.empty((self.cfg.n_obstacles, 10, self.n), dtype=torch.float32, device=self.device)
        _abi.ag_get_obstacles(self.ctx, out)
        return out

    def set_obstacle_randomization(self, env_min, env_max, per_box) -> None:
        """per_box: list of _abi.ag_box_randomization (one per obstacle), or None to disable."""
        _abi.ag_set_obstacle_randomization(self.ctx, env_min, env_max, per_box)

    def render_depth(self, width: int, height: int, hfov: float, max_range: float, cam_offset=None,
                     env_ids=None, n_cams: int | None = None, out=None) -> torch.Tensor:
        """float32 [n_cams, height, width] depth images (see ag_render_depth)."""
        ids = None if env_ids is None else self._dev(env_ids, torch.int32)
        n_cams = (self.n if ids is None else ids.numel()) if n_cams is None else n_cams
        if out is None:
            out = torch.empty((n_cams, height, width), dtype=torch.float32, device=self.device)
        _abi.ag_render_depth(self.ctx, width, height, hfov, max_range, cam_offset, ids, n_cams, out)
        self._keep_ids = ids
        return out

    def eval_controller(self, state=None) -> torch.Tensor:
        """float32 [4, n] commanded (f, M_x, M_y, M_z) of every environment's
        controller at `state` [13, n] (None = the current states); see ag_eval_controller."""
        s = None if state is None else self._dev(state, torch.float32)
        out = torch.empty((4, self.n), dtype=torch.float32, device=self.device)
        _abi.ag_eval_controller(self.ctx, s, out)
        self._keep_eval = s
        return out

    def set_body(self, body) -> None:
        b = self._dev(body, torch.float32)
        _abi.ag_set_body(self.ctx, b)
        self._keep_body = b

    # ---------------------------------------------------------------- steps --
    def step(self, n_steps: int = 1) -> None:
        _abi.ag_step(self.ctx, n_steps * self.cfg.substeps_per_step)

    def step_plain(self, n_steps: int = 1) -> None:
        _abi.ag_step_plain(self.ctx, n_steps * self.cfg.substeps_per_step)

    def reset(self, mask=None, seed: int | None = None) -> None:
        m = None if mask is None else self._dev(mask, torch.uint8)
        _abi.ag_reset(self.ctx, m, self.cfg.seed if seed is None else seed)
        self._keep_mask = m

    # -------------------------------------------------------------- outputs --
    def state(self) -> torch.Tensor:
        out = torch.empty((13, self.n), dtype=torch.float32, device=self.device)
        _abi.ag_get_state(self.ctx, state=out)
        return out

    def motors(self) -> torch.Tensor:
        out = torch.empty((8, self.n), dtype=torch.float32, device=self.device)
        _abi.ag_get_motors(self.ctx, motors=out)
        return out

    def epoch(self) -> torch.Tensor:
        out = torch.empty((self.n,), dtype=torch.int32, device=self.device)
        _abi.ag_get_motors(self.ctx, epoch=out)
        return out

    def events(self):
        """(collided uint8[n], reset ids of the last call as an int64 tensor)."""
        col = torch.empty((self.n,), dtype=torch.uint8, device=self.device)
        ids = torch.empty((self.n,), dtype=torch.int32, device=self.device)
        cnt = _abi.ag_get_state(self.ctx, collided=col, reset_ids=ids, want_count=True)
        return col, ids[:cnt].to(torch.int64)

    def set_state(self, state, motors=None, epoch=None) -> None:
        s = self._dev(state, torch.float32)
        m = None if motors is None else self._dev(motors, torch.float32)
        e = None if epoch is None else self._dev(epoch, torch.int32)
        _abi.ag_set_state(self.ctx, s, m, e)
        self._keep_state = (s, m, e)

    def synchronize(self) -> None:
        _abi.ag_synchronize(self.ctx)
