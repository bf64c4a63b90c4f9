"""The allocation-free unfused step against the context-based one.

ag_step_plain_noalloc serves callers that may not allocate device memory
(a simulator inside a real-time control loop, where cudaMalloc's device
synchronisation and latency are not allowed once the loop runs, or a host
application that owns the whole device-memory budget). It keeps its scratch
in a static device array shared by every call, so this file runs last: if
it fails, a run that stops at the first failure has already run every other
test. It must pass alone in a fresh process and after the other tests.
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


def test_noalloc_step_matches_context_step_on_two_calls():
    w = W.scaled(W.WORKLOADS["obstacles"], 5000)
    seed = 17
    inp = W.make_inputs(w, seed)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    cfg = _config(w, seed)
    ctx = _abi.ag_create(cfg, stream.cuda_stream)
    try:
        modes = torch.from_numpy(inp.modes).to(dev)
        targets = torch.from_numpy(inp.targets).to(dev)
        body = torch.from_numpy(inp.body).to(dev)
        boxes = torch.from_numpy(inp.boxes).to(dev)
        _abi.ag_set_body(ctx, body)
        _abi.ag_set_commands(ctx, modes, targets)
        _abi.ag_set_obstacles(ctx, boxes)
        _abi.ag_reset(ctx, None, seed)
        n = w.n_envs
        # the caller's own buffers for the allocation-free call, same start
        state = torch.empty((13, n), dtype=torch.float32, device=dev)
        motors = torch.empty((8, n), dtype=torch.float32, device=dev)
        epoch = torch.empty((n,), dtype=torch.int32, device=dev)
        _abi.ag_get_state(ctx, state=state)
        _abi.ag_get_motors(ctx, motors=motors, epoch=epoch)
        collided = torch.empty((n,), dtype=torch.uint8, device=dev)
        reset_ids = torch.empty((n,), dtype=torch.int32, device=dev)
        n_reset = torch.empty((1,), dtype=torch.int32, device=dev)
        n_sub = 25 * w.substeps_per_step
        total_resets = 0
        for _ in range(2):
            _abi.ag_step_plain(ctx, n_sub)
            _abi.ag_step_plain_noalloc(cfg, stream.cuda_stream, n_sub, seed, state, motors, body, modes, targets,
                                       boxes, epoch, collided, reset_ids, n_reset)
            ref_state = torch.empty_like(state)
            ref_motors = torch.empty_like(motors)
            ref_epoch = torch.empty_like(epoch)
            ref_col = torch.empty_like(collided)
            ref_ids = torch.empty_like(reset_ids)
            _abi.ag_get_motors(ctx, motors=ref_motors, epoch=ref_epoch)
            ref_n = _abi.ag_get_state(ctx, state=ref_state, collided=ref_col, reset_ids=ref_ids, want_count=True)
            torch.cuda.synchronize()
            np.testing.assert_allclose(state.cpu().numpy(), ref_state.cpu().numpy(), atol=1e-5, rtol=1e-6)
            np.testing.assert_allclose(motors.cpu().numpy(), ref_motors.cpu().numpy(), atol=1e-5, rtol=1e-6)
            np.testing.assert_array_equal(epoch.cpu().numpy(), ref_epoch.cpu().numpy())
            np.testing.assert_array_equal(collided.cpu().numpy(), ref_col.cpu().numpy())
            got_n = int(n_reset.item())
            assert got_n == ref_n
            assert sorted(reset_ids[:got_n].cpu().tolist()) == sorted(ref_ids[:ref_n].cpu().tolist())
            total_resets += got_n
        assert total_resets > 0          # the collision/reset stage really ran
    finally:
        _abi.ag_destroy(ctx)


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
