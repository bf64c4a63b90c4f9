"""The hand-written adjoint (ag_backward) against the FP64 oracle.

Workload: 65,536 quads in position mode, semi-implicit Euler, 256 steps,
loss = sum_t |p_t - p_goal|^2 + 0.01 |Omega_t|^2, checkpoint every 32 steps.
Gradients with respect to the initial state (13 per vehicle) and the 12
gains are compared with FP64 central finite differences of the oracle's loss
on 64 sampled vehicles (relative error <= 1e-3) and with the oracle's
forward-mode (dual-number) directional derivative. Where a motor clamp
switches inside the finite-difference step the loss has a kink there: a
component whose one-sided differences keep the same gap when the step is
halved is such a kink and is excluded (and counted); a second workload with
small errors, where no motor ever saturates, must match on every component.
"""
import numpy as np
import pytest
import torch

import oracle as O
from harness import gpu_fleet, oracle_world
from paper_2305_16510_gb300 import _abi
from paper_2305_16510_gb300 import workloads as W

pytestmark = pytest.mark.gpu
H, W_POS, W_OMEGA = 256, 1.0, 0.01
GAINS = np.array([2, 2, 3, 2, 2, 2, 1.2, 1.2, 0.6, 0.2, 0.2, 0.1], dtype=np.float64)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2305_16510_gb300 import build
    build.build()


def _np(t):
    return t.detach().cpu().numpy()


def _run(w, inp, seed, gentle=False):
    fl = gpu_fleet(w, inp, seed)
    fl.reset(None, seed)
    if gentle:
        # start within 0.3 m of the target, level, at rest, yaw at the target
        st = _np(fl.state())
        st[0:3] = inp.targets[0:3] + 0.3 * np.random.default_rng(seed).uniform(-1, 1, (3, w.n_envs))
        st[3:6] = 0.0
        half = 0.5 * inp.targets[3]
        st[6], st[7], st[8], st[9] = np.cos(half), 0.0, 0.0, np.sin(half)
        st[10:13] = 0.0
        fl.set_state(st.astype(np.float32))
    x0, m0 = _np(fl.state()), _np(fl.motors())
    n = w.n_envs
    goal = torch.from_numpy(np.ascontiguousarray(inp.targets[0:3])).cuda()
    loss = torch.empty(n, dtype=torch.float32, device="cuda")
    sat = torch.empty(n, dtype=torch.uint8, device="cuda")
    _abi.ag_rollout_loss(fl.ctx, H, W_POS, W_OMEGA, goal, loss, sat)
    gx = torch.empty((13, n), dtype=torch.float32, device="cuda")
    gg = torch.empty((12,), dtype=torch.float32, device="cuda")
    gge = torch.empty((12, n), dtype=torch.float32, device="cuda")
    _abi.ag_backward(fl.ctx, None, gx, gg, gge)
    torch.cuda.synchronize()
    return fl, x0, m0, _np(loss), _np(sat), _np(gx), _np(gg), _np(gge), goal


def _oracle_loss(world, i, inp, x0, m0, gains, s=None):
    state = x0[:, i].astype(np.float64) if s is None else s
    return O.vehicle_loss(world, 4, O.MODE_POSITION, inp.targets[:, i].astype(np.float64),
                          inp.body[:, i].astype(np.float64), state, m0[0:4, i].astype(np.float64), gains, H,
                          inp.targets[0:3, i].astype(np.float64), W_POS, W_OMEGA)


def _fd_gradient(world, i, inp, x0, m0, detect_kinks):
    """Central differences of the FP64 oracle loss: (grad[25], smooth[25]).

    With detect_kinks, a component is a kink when the gap between its
    one-sided differences does not halve with the step (a smooth function's
    gap is h f'' and halves; a slope jump inside the step does not)."""
    base = np.concatenate([x0[:, i].astype(np.float64), GAINS])
    L0 = _oracle_loss(world, i, inp, x0, m0, GAINS) if detect_kinks else None
    g = np.zeros(25)
    smooth = np.ones(25, bool)

    def at(k, delta):
        v = base.copy()
        v[k] += delta
        return _oracle_loss(world, i, inp, x0, m0, v[13:], s=v[:13])

    for k in range(25):
        h = 1e-6 * max(1.0, abs(base[k]))
        lp, lm = at(k, h), at(k, -h)
        g[k] = (lp - lm) / (2 * h)
        if detect_kinks:
            gap1 = (lp - L0) / h - (L0 - lm) / h
            lp2, lm2 = at(k, h / 2), at(k, -h / 2)
            gap2 = (lp2 - L0) / (h / 2) - (L0 - lm2) / (h / 2)
            smooth[k] = abs(gap2 - 0.5 * gap1) <= 0.25 * abs(gap1) + 1e-6 * max(1.0, abs(g[k]))
    return g, smooth


def _compare(w, inp, seed, gentle):
    fl, x0, m0, loss, sat, gx, gg, gge, _ = _run(w, inp, seed, gentle)
    fl.close()
    world = oracle_world(w)
    idx = np.sort(np.random.default_rng(seed).choice(w.n_envs, 64, replace=False))
    kinks = 0
    for i in idx:
        L = _oracle_loss(world, i, inp, x0, m0, GAINS)
        assert abs(loss[i] - L) <= 1e-4 * max(1.0, abs(L)), (i, loss[i], L)
        g_fd, smooth = _fd_gradient(world, i, inp, x0, m0, detect_kinks=not gentle)
        g_gpu = np.concatenate([gx[:, i], gge[:, i]]).astype(np.float64)
        kinks += int((~smooth).sum())
        err = np.linalg.norm((g_gpu - g_fd)[smooth]) / max(np.linalg.norm(g_fd[smooth]), 1e-6)
        assert err <= 1e-3, (i, err, g_gpu, g_fd)
    return kinks, sat


def test_adjoint_matches_fd_on_the_adjoint_workload():
    w = W.WORKLOADS["adjoint"]
    inp = W.make_inputs(w, 5)
    kinks, sat = _compare(w, inp, 5, gentle=False)
    assert kinks <= 64 * 25 // 10      # kinks are the exception, not the rule
    assert sat.mean() > 0.0            # the workload does exercise the clamp


def test_adjoint_matches_fd_every_component_without_saturation():
    w = W.scaled(W.WORKLOADS["adjoint"], 4096)
    inp = W.make_inputs(w, 6)
    kinks, sat = _compare(w, inp, 6, gentle=True)
    assert sat.sum() == 0              # no clamp anywhere: every component is compared
    assert kinks == 0


def test_adjoint_matches_oracle_dual_number_jvp():
    w = W.scaled(W.WORKLOADS["adjoint"], 2048)
    inp = W.make_inputs(w, 7)
    fl, x0, m0, loss, sat, gx, gg, gge, _ = _run(w, inp, 7)
    fl.close()
    world = oracle_world(w)
    rng = np.random.default_rng(8)
    for i in rng.choice(w.n_envs, 16, replace=False):
        ds, dgn = rng.normal(size=13), rng.normal(size=12)
        _, jvp = O.vehicle_loss_jvp(world, 4, O.MODE_POSITION, inp.targets[:, i].astype(np.float64),
                                    inp.body[:, i].astype(np.float64), x0[:, i].astype(np.float64),
                                    m0[0:4, i].astype(np.float64), GAINS, ds, dgn, H,
                                    inp.targets[0:3, i].astype(np.float64), W_POS, W_OMEGA)
        dot = float(gx[:, i].astype(np.float64) @ ds + gge[:, i].astype(np.float64) @ dgn)
        assert abs(dot - jvp) <= 1e-3 * max(1.0, abs(jvp)), (i, dot, jvp)


def test_gain_gradient_reduction_is_deterministic_and_weighted():
    w = W.WORKLOADS["adjoint"]
    inp = W.make_inputs(w, 9)
    fl, x0, m0, loss, sat, gx, gg, gge, goal = _run(w, inp, 9)
    n = w.n_envs
    gg2 = torch.empty(12, dtype=torch.float32, device="cuda")
    _abi.ag_backward(fl.ctx, None, None, gg2, None)
    assert np.array_equal(_np(gg2), gg)                       # bit-identical repeat
    np.testing.assert_allclose(gg, gge.astype(np.float64).sum(axis=1), rtol=1e-4, atol=1e-3)
    wts = torch.from_numpy(np.random.default_rng(1).uniform(0, 2, n).astype(np.float32)).cuda()
    gxw = torch.empty((13, n), dtype=torch.float32, device="cuda")
    ggew = torch.empty((12, n), dtype=torch.float32, device="cuda")
    _abi.ag_backward(fl.ctx, wts, gxw, None, ggew)
    np.testing.assert_allclose(_np(gxw), gx * _np(wts)[None, :], rtol=1e-5, atol=1e-6 * np.abs(gx).max())
    np.testing.assert_allclose(_np(ggew), gge * _np(wts)[None, :], rtol=1e-5, atol=1e-6 * np.abs(gge).max())
    fl.close()


def test_autograd_function_matches_ag_backward():
    from paper_2305_16510_gb300.autograd import rollout_loss
    w = W.scaled(W.WORKLOADS["adjoint"], 1024)
    inp = W.make_inputs(w, 10)
    fl, x0, m0, loss, sat, gx, gg, gge, goal = _run(w, inp, 10)
    x0_t = torch.from_numpy(x0).cuda().requires_grad_(True)
    gains_t = torch.tensor(GAINS, dtype=torch.float32, requires_grad=True)
    m0_t = torch.from_numpy(m0).cuda()
    out = rollout_loss(fl, x0_t, gains_t, m0_t, H, goal, W_POS, W_OMEGA)
    np.testing.assert_allclose(_np(out), loss, rtol=1e-6)
    out.sum().backward()
    np.testing.assert_allclose(_np(x0_t.grad), gx, rtol=1e-6, atol=1e-6 * np.abs(gx).max())
    np.testing.assert_allclose(_np(gains_t.grad), gg, rtol=1e-6)
    fl.close()


def test_unsupported_configurations_are_refused():
    w = W.Workload("rk4", 256, 4, 1, 0, 256, 0, 0)
    inp = W.make_inputs(w, 1)
    fl = gpu_fleet(w, inp, 1)
    goal = torch.zeros((3, 256), device="cuda")
    loss = torch.empty(256, device="cuda")
    with pytest.raises(_abi.AgError) as e:
        _abi.ag_rollout_loss(fl.ctx, 10, 1.0, 0.01, goal, loss)
    assert e.value.status == _abi.AG_ERR_UNSUPPORTED
    with pytest.raises(_abi.AgError) as e:
        _abi.ag_backward(fl.ctx, None, torch.empty((13, 256), device="cuda"))
    assert e.value.status == _abi.AG_ERR_STATE
    fl.close()
    w = W.Workload("vel", 256, 1, 0, 0, 256, 0, 0, mode_mix=(W.MODE_BODY_VEL,))
    fl = gpu_fleet(w, W.make_inputs(w, 1), 1)
    with pytest.raises(_abi.AgError) as e:
        _abi.ag_rollout_loss(fl.ctx, 10, 1.0, 0.01, goal, loss)
    assert e.value.status == _abi.AG_ERR_UNSUPPORTED
    fl.close()
