"""The allocation-free unfused step against the context-based one.

ag_step_plain_noalloc serves callers that may not allocate device memory
(a simulator inside a real-time control loop, where cudaMalloc's device
synchronisation and latency are not allowed once the loop runs, or a host
application that owns the whole device-memory budget). It keeps its scratch
in a static device array shared by every call, so this file runs last: if
it fails, a run that stops at the first failure has already run every other
test. It must pass alone in a fresh process and after the other tests.

Both entry points launch the same stage kernels with the same parameters on
the same inputs, so their results must agree bit for bit.
"""
import numpy as np
import pytest
import torch

from paper_2305_16510_gb300 import _abi
from paper_2305_16510_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2305_16510_gb300 import build
    build.build()


def _config(w, seed):
    c = _abi.ag_config_default()
    c.n_envs, c.substeps_per_step, c.integrator, c.n_obstacles = w.n_envs, w.substeps_per_step, w.integrator, \
        w.n_obstacles
    c.n_quad, c.n_hexa, c.n_octo = w.n_quad, w.n_hexa, w.n_octo
    c.motor_tau, c.drag, c.seed = w.motor_tau, w.drag, seed
    return c


class _Pair:
    """A context and the caller-owned buffers of the allocation-free call,
    both starting from the context's Philox reset."""

    def __init__(self, w, seed):
        self.w, self.seed = w, seed
        inp = W.make_inputs(w, seed)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.stream = torch.cuda.current_stream()
        self.cfg = _config(w, seed)
        self.ctx = _abi.ag_create(self.cfg, self.stream.cuda_stream)
        self.modes = torch.from_numpy(inp.modes).to(dev)
        self.targets = torch.from_numpy(inp.targets).to(dev)
        self.body = torch.from_numpy(inp.body).to(dev)
        self.boxes = None if inp.boxes is None else torch.from_numpy(inp.boxes).to(dev)
        _abi.ag_set_body(self.ctx, self.body)
        _abi.ag_set_commands(self.ctx, self.modes, self.targets)
        if self.boxes is not None:
            _abi.ag_set_obstacles(self.ctx, self.boxes)
        _abi.ag_reset(self.ctx, None, seed)
        n = w.n_envs
        self.state = torch.empty((13, n), dtype=torch.float32, device=dev)
        self.motors = torch.empty((8, n), dtype=torch.float32, device=dev)
        self.epoch = torch.empty((n,), dtype=torch.int32, device=dev)
        _abi.ag_get_state(self.ctx, state=self.state)
        _abi.ag_get_motors(self.ctx, motors=self.motors, epoch=self.epoch)
        self.collided = torch.empty((n,), dtype=torch.uint8, device=dev)
        self.reset_ids = torch.empty((n,), dtype=torch.int32, device=dev)
        self.n_reset = torch.empty((1,), dtype=torch.int32, device=dev)

    def step_noalloc(self, n_sub):
        _abi.ag_step_plain_noalloc(self.cfg, self.stream.cuda_stream, n_sub, self.seed, self.state, self.motors,
                                   self.body, self.modes, self.targets, self.boxes, self.epoch, self.collided,
                                   self.reset_ids, self.n_reset)

    def check_equal(self):
        """Both sides bit for bit; returns this call's reset count."""
        ref_state = torch.empty_like(self.state)
        ref_motors = torch.empty_like(self.motors)
        ref_epoch = torch.empty_like(self.epoch)
        ref_col = torch.empty_like(self.collided)
        ref_ids = torch.empty_like(self.reset_ids)
        _abi.ag_get_motors(self.ctx, motors=ref_motors, epoch=ref_epoch)
        ref_n = _abi.ag_get_state(self.ctx, state=ref_state, collided=ref_col, reset_ids=ref_ids, want_count=True)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(self.state.cpu().numpy(), ref_state.cpu().numpy())
        np.testing.assert_array_equal(self.motors.cpu().numpy(), ref_motors.cpu().numpy())
        np.testing.assert_array_equal(self.epoch.cpu().numpy(), ref_epoch.cpu().numpy())
        np.testing.assert_array_equal(self.collided.cpu().numpy(), ref_col.cpu().numpy())
        got_n = int(self.n_reset.item())
        assert got_n == ref_n
        # the reset list's order depends on warp scheduling; its contents do not
        assert sorted(self.reset_ids[:got_n].cpu().tolist()) == sorted(ref_ids[:ref_n].cpu().tolist())
        return got_n

    def close(self):
        _abi.ag_destroy(self.ctx)


def test_noalloc_step_matches_context_step_on_two_calls():
    pair = _Pair(W.scaled(W.WORKLOADS["obstacles"], 5000), 17)
    try:
        n_sub = 25 * pair.w.substeps_per_step
        total_resets = 0
        for _ in range(2):
            _abi.ag_step_plain(pair.ctx, n_sub)
            pair.step_noalloc(n_sub)
            total_resets += pair.check_equal()
        assert total_resets > 0          # the collision/reset stage really ran
    finally:
        pair.close()


def test_noalloc_at_its_maximum_fleet_size_allocates_nothing():
    """Exactly AG_NOALLOC_MAX_ENVS environments (the size the static array is
    laid out for), a short horizon, two calls; after a warm-up call, a call
    changes neither the device's free memory nor torch's reserved bytes."""
    n = _abi.AG_NOALLOC_MAX_ENVS
    pair = _Pair(W.scaled(W.WORKLOADS["obstacles"], n), 23)
    try:
        n_sub = 3 * pair.w.substeps_per_step
        total_resets = 0
        for _ in range(2):
            _abi.ag_step_plain(pair.ctx, n_sub)
            pair.step_noalloc(n_sub)
            total_resets += pair.check_equal()
        assert total_resets > 0
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        reserved0 = torch.cuda.memory_reserved()
        pair.step_noalloc(n_sub)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        assert torch.cuda.memory_reserved() == reserved0
    finally:
        pair.close()


def test_noalloc_rejects_more_envs_than_its_scratch_holds():
    w = W.Workload("big", _abi.AG_NOALLOC_MAX_ENVS + 1, 1, 0, 0, _abi.AG_NOALLOC_MAX_ENVS + 1, 0, 0)
    cfg = _config(w, 1)
    dev = torch.device("cuda", torch.cuda.current_device())
    n = w.n_envs
    buf = torch.zeros((16, n), dtype=torch.float32, device=dev)
    with pytest.raises(_abi.AgError) as e:
        _abi.ag_step_plain_noalloc(cfg, None, 1, 1, buf, buf, buf, buf, buf, None, buf, buf, buf, buf)
    assert e.value.status == _abi.AG_ERR_INVALID
    assert "AG_NOALLOC_MAX_ENVS" in str(e.value)


def test_noalloc_rejects_buffers_the_current_device_cannot_use():
    """Host memory, and (with a second GPU) another device's memory or stream,
    are refused before anything is launched."""
    w = W.Workload("small", 256, 1, 0, 0, 256, 0, 0)
    cfg = _config(w, 1)
    dev = torch.device("cuda", torch.cuda.current_device())
    buf = torch.zeros((16, 256), dtype=torch.float32, device=dev)
    host = torch.zeros((16, 256), dtype=torch.float32).pin_memory()
    with pytest.raises(_abi.AgError) as e:
        _abi.ag_step_plain_noalloc(cfg, None, 1, 1, buf, host, buf, buf, buf, None, buf, buf, buf, buf)
    assert e.value.status == _abi.AG_ERR_INVALID
    if torch.cuda.device_count() > 1:
        other = (torch.cuda.current_device() + 1) % torch.cuda.device_count()
        far = torch.zeros((16, 256), dtype=torch.float32, device=torch.device("cuda", other))
        with pytest.raises(_abi.AgError) as e:
            _abi.ag_step_plain_noalloc(cfg, None, 1, 1, buf, far, buf, buf, buf, None, buf, buf, buf, buf)
        assert e.value.status == _abi.AG_ERR_INVALID
        with torch.cuda.device(other):
            far_stream = torch.cuda.Stream()
        with pytest.raises(_abi.AgError) as e:
            _abi.ag_step_plain_noalloc(cfg, far_stream.cuda_stream, 1, 1, buf, buf, buf, buf, buf, None, buf, buf,
                                       buf, buf)
        assert e.value.status == _abi.AG_ERR_INVALID
