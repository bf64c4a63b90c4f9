"""Python face of the continuous-batching rollout server (ag_server_*).

The server loop itself is native (serve.cu): admission, batching, launches
and retirement all run in the library's host thread and kernels. This module
only builds request descriptors over torch tensors and collects results.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _abi


class RequestPool:
    """Device-resident input arrays that requests take slices of.

    modes uint8 [N], targets float32 [4, N], boxes float32 [n_obs_max * 10, N]
    (or None). A request of n envs at offset o uses columns o .. o + n - 1 and
    its first n_obstacles boxes (row stride N).
    """

    def __init__(self, modes, targets, boxes=None, body=None, device=None):
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.modes = torch.as_tensor(modes).to(dev, torch.uint8).contiguous()
        self.targets = torch.as_tensor(targets).to(dev, torch.float32).contiguous()
        self.boxes = None if boxes is None else torch.as_tensor(boxes).to(dev, torch.float32).reshape(
            -1, self.modes.numel()).contiguous()
        self.body = None if body is None else torch.as_tensor(body).to(dev, torch.float32).contiguous()
        self.N = self.modes.numel()

    def request(self, n_envs: int, n_steps: int, n_obstacles: int, seed: int, offset: int = 0) -> _abi.ag_request:
        if offset + n_envs > self.N:
            raise ValueError("request slice exceeds the pool")
        r = _abi.ag_request()
        r.n_envs, r.n_steps, r.n_obstacles, r.seed = n_envs, n_steps, n_obstacles, seed
        r.modes = self.modes.data_ptr() + offset
        r.targets = self.targets.data_ptr() + 4 * offset
        r.body = None if self.body is None else self.body.data_ptr() + 4 * offset
        r.boxes = None if (n_obstacles == 0 or self.boxes is None) else self.boxes.data_ptr() + 4 * offset
        r.pitch = self.N
        return r


class Server:
    """One ag_server. submit() is non-blocking; wait() returns (state, epoch, latency_ms)."""

    def __init__(self, *, max_active: int = 1024, chunk_steps: int = 50, hbm_budget_bytes: int = 40 << 30,
                 integrator: int = _abi.AG_INTEG_RK4, substeps_per_step: int = 4, **physics):
        c = _abi.ag_server_config_default()
        c.max_active, c.chunk_steps, c.hbm_budget_bytes = max_active, chunk_steps, hbm_budget_bytes
        c.physics.integrator, c.physics.substeps_per_step = integrator, substeps_per_step
        for k, v in physics.items():
            setattr(c.physics, k, v)
        self.cfg = c
        self.handle = _abi.ag_server_create(c)
        self._sizes = {}

    def submit(self, req: _abi.ag_request) -> int:
        rid = _abi.ag_server_submit(self.handle, req)
        self._sizes[rid] = req.n_envs
        return rid

    def wait(self, rid: int, timeout_s: float = 600.0, want_state: bool = True):
        n = self._sizes[rid]
        st = np.empty((13, n), np.float32) if want_state else None
        ep = np.empty(n, np.uint32) if want_state else None
        lat = _abi.ag_server_wait(self.handle, rid, timeout_s, st, ep)
        del self._sizes[rid]
        return st, ep, lat

    def stats(self) -> _abi.ag_server_stats:
        return _abi.ag_server_get_stats(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            _abi.ag_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
