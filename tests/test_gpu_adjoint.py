"""The hand-written adjoint (ag_backward) against the FP64 oracle.

Main workload: 65,536 quads in position mode, semi-implicit Euler, 256 steps,
loss = sum_t |p_t - p_goal|^2 + 0.01 |Omega_t|^2, checkpoint every 32 steps.
Gradients with respect to the initial state (13 per vehicle) and the 12
gains are compared with FP64 central finite differences of the oracle's loss
on 64 sampled vehicles (relative error <= 1e-3) and with the oracle's
forward-mode (dual-number) directional derivative. Where a motor clamp
switches inside the finite-difference step the loss has a kink there: a
component whose one-sided differences keep the same gap when the step is
halved is such a kink and is excluded (and counted); a second workload with
small errors, where no motor ever saturates, must match on every component.
The other command modes (body velocity, attitude and thrust, wrench) and
hexa / octo rotors are checked the same way, including the gradient with
respect to each environment's four command targets.
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
    worst = 0.0
    for i in idx:
        L = _oracle_loss(world, i, inp, x0, m0, GAINS)
        assert abs(loss[i] - L) <= 1e-4 * max(1.0, abs(L)), (i, loss[i], L)
        g_fd, smooth = _fd_gradient(world, i, inp, x0, m0, detect_kinks=not gentle)
        g_gpu = np.concatenate([gx[:, i], gge[:, i]]).astype(np.float64)
        kinks += int((~smooth).sum())
        err = np.linalg.norm((g_gpu - g_fd)[smooth]) / max(np.linalg.norm(g_fd[smooth]), 1e-6)
        assert err <= 1e-3, (i, err, g_gpu, g_fd)
        worst = max(worst, err)
    return kinks, sat, worst


def test_adjoint_matches_fd_on_the_adjoint_workload(within_tolerance):
    w = W.WORKLOADS["adjoint"]
    inp = W.make_inputs(w, 5)
    kinks, sat, worst = _compare(w, inp, 5, gentle=False)
    # the gradient bar of the differentiable-rollout workload
    within_tolerance("|g - g_fd| / |g_fd| (64 vehicles, kinks excluded)", worst, 1e-3)
    assert kinks <= 64 * 25 // 10      # kinks are the exception, not the rule
    assert sat.mean() > 0.0            # the workload does exercise the clamp


def test_adjoint_matches_fd_every_component_without_saturation(within_tolerance):
    w = W.scaled(W.WORKLOADS["adjoint"], 4096)
    inp = W.make_inputs(w, 6)
    kinks, sat, worst = _compare(w, inp, 6, gentle=True)
    within_tolerance("|g - g_fd| / |g_fd| (64 vehicles, every component)", worst, 1e-3)
    assert sat.sum() == 0              # no clamp anywhere: every component is compared
    assert kinks == 0


def test_adjoint_matches_oracle_dual_number_jvp(within_tolerance):
    w = W.scaled(W.WORKLOADS["adjoint"], 2048)
    inp = W.make_inputs(w, 7)
    fl, x0, m0, loss, sat, gx, gg, gge, _ = _run(w, inp, 7)
    fl.close()
    world = oracle_world(w)
    rng = np.random.default_rng(8)
    worst = 0.0
    for i in rng.choice(w.n_envs, 16, replace=False):
        ds, dgn = rng.normal(size=13), rng.normal(size=12)
        _, jvp = O.vehicle_loss_jvp(world, 4, O.MODE_POSITION, inp.targets[:, i].astype(np.float64),
                                    inp.body[:, i].astype(np.float64), x0[:, i].astype(np.float64),
                                    m0[0:4, i].astype(np.float64), GAINS, ds, dgn, H,
                                    inp.targets[0:3, i].astype(np.float64), W_POS, W_OMEGA)
        dot = float(gx[:, i].astype(np.float64) @ ds + gge[:, i].astype(np.float64) @ dgn)
        assert abs(dot - jvp) <= 1e-3 * max(1.0, abs(jvp)), (i, dot, jvp)
        worst = max(worst, abs(dot - jvp) / max(1.0, abs(jvp)))
    within_tolerance("|g . d - JVP| / max(1, |JVP|) (16 vehicles)", worst, 1e-3)


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
    # a second recording on the same fleet: the first loss's backward refuses, the second's works
    xa = torch.from_numpy(x0).cuda().requires_grad_(True)
    xb = torch.from_numpy(x0).cuda().requires_grad_(True)
    out_a = rollout_loss(fl, xa, gains_t.detach(), m0_t, H, goal, W_POS, W_OMEGA)
    out_b = rollout_loss(fl, xb, gains_t.detach(), m0_t, H, goal, W_POS, W_OMEGA)
    with pytest.raises(RuntimeError, match="recorded another rollout"):
        out_a.sum().backward()
    out_b.sum().backward()
    np.testing.assert_allclose(_np(xb.grad), gx, rtol=1e-6, atol=1e-6 * np.abs(gx).max())
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
    w = W.Workload("obs", 256, 1, 0, 2, 256, 0, 0)
    fl = gpu_fleet(w, W.make_inputs(w, 1), 1)
    with pytest.raises(_abi.AgError) as e:
        _abi.ag_rollout_loss(fl.ctx, 10, 1.0, 0.01, goal, loss)
    assert e.value.status == _abi.AG_ERR_UNSUPPORTED
    fl.close()


# --------------------------------------------------- every command mode --
H_MODES = 96
MODE_NAMES = {W.MODE_POSITION: "position", W.MODE_BODY_VEL: "velocity", W.MODE_ATT_THRUST: "attitude",
              W.MODE_WRENCH: "wrench"}


def _mode_inputs(w, seed, gentle):
    """Inputs of every mode; gentle keeps each motor well inside [0, u_max]."""
    inp = W.make_inputs(w, seed)
    rng = np.random.default_rng(seed + 100)
    m = inp.body[0].astype(np.float64)
    t = inp.targets.astype(np.float64)
    for i in range(w.n_envs):
        md = inp.modes[i]
        if md == W.MODE_WRENCH:
            t[:, i] = [m[i] * 9.81 * rng.uniform(0.97, 1.03), *rng.uniform(-2e-3, 2e-3, 3)]
        elif gentle and md == W.MODE_ATT_THRUST:
            t[:, i] = [*rng.uniform(-0.15, 0.15, 2), rng.uniform(-0.5, 0.5), m[i] * 9.81 * rng.uniform(0.95, 1.05)]
        elif gentle and md == W.MODE_BODY_VEL:
            t[:, i] = [*rng.uniform(-0.5, 0.5, 3), rng.uniform(-0.3, 0.3)]
        elif gentle and md == W.MODE_POSITION:
            t[:, i] = [*rng.uniform(-0.5, 0.5, 3), rng.uniform(-np.pi, np.pi)]
    return W.Inputs(inp.modes, t.astype(np.float32), inp.body, None)


def _run_modes(w, inp, seed, gentle):
    fl = gpu_fleet(w, inp, seed)
    fl.reset(None, seed)
    if gentle:   # level, at rest, yaw U[-pi, pi); position-mode vehicles within 0.3 m of their target
        rng = np.random.default_rng(seed)
        st = _np(fl.state())
        pos = inp.modes == W.MODE_POSITION
        st[0:3, pos] = inp.targets[0:3, pos] + rng.uniform(-0.3, 0.3, (3, int(pos.sum())))
        st[3:6] = 0.0
        st[10:13] = 0.0
        yaw = rng.uniform(-np.pi, np.pi, w.n_envs)
        # yaw authority is small (k_yaw = 0.016): a yaw error of 0.2 rad already drives a motor to 0
        yaw[pos] = inp.targets[3, pos] + rng.uniform(-0.05, 0.05, int(pos.sum()))
        half = yaw / 2
        st[6], st[7], st[8], st[9] = np.cos(half), 0.0, 0.0, np.sin(half)
        fl.set_state(st.astype(np.float32))
    x0, m0 = _np(fl.state()), _np(fl.motors())
    n = w.n_envs
    goal = (x0[0:3] + 0.2 * np.random.default_rng(seed + 1).uniform(-1, 1, (3, n))).astype(np.float32)
    loss = torch.empty(n, device="cuda")
    sat = torch.empty(n, dtype=torch.uint8, device="cuda")
    _abi.ag_rollout_loss(fl.ctx, H_MODES, W_POS, W_OMEGA, torch.from_numpy(goal).cuda(), loss, sat)
    gx = torch.empty((13, n), device="cuda")
    gge = torch.empty((12, n), device="cuda")
    gt = torch.empty((4, n), device="cuda")
    _abi.ag_backward(fl.ctx, None, gx, None, gge, gt)
    torch.cuda.synchronize()
    fl.close()
    return x0, m0, goal, _np(loss), _np(sat), _np(gx), _np(gge), _np(gt)


def _rotors(w, i):
    return 4 if i < w.n_quad else (6 if i < w.n_quad + w.n_hexa else 8)


def _loss29(world, w, inp, i, x0, m0, goal, v):
    """Oracle loss at v = (x0 (13), gains (12), targets (4))."""
    nr = _rotors(w, i)
    return O.vehicle_loss(world, nr, int(inp.modes[i]), v[25:29], inp.body[:, i].astype(np.float64), v[:13],
                          m0[0:nr, i].astype(np.float64), v[13:25], H_MODES, goal[:, i].astype(np.float64), W_POS,
                          W_OMEGA)


def _sample(w, inp, per_cell, seed):
    rng = np.random.default_rng(seed)
    out = []
    for md in MODE_NAMES:
        for lo, hi in [(0, w.n_quad), (w.n_quad, w.n_quad + w.n_hexa), (w.n_quad + w.n_hexa, w.n_envs)]:
            cand = np.nonzero(inp.modes[lo:hi] == md)[0] + lo
            out += list(rng.choice(cand, min(per_cell, len(cand)), replace=False))
    return sorted(out)


MODES_W = W.Workload("modes", 3072, 1, 0, 0, 1024, 1024, 1024, drag=0.1, horizon=H_MODES,
                     mode_mix=(W.MODE_POSITION, W.MODE_BODY_VEL, W.MODE_ATT_THRUST, W.MODE_WRENCH))


def test_adjoint_every_mode_matches_oracle_jvp_with_target_tangents():
    w = MODES_W
    inp = _mode_inputs(w, 21, gentle=False)
    x0, m0, goal, loss, sat, gx, gge, gt = _run_modes(w, inp, 21, gentle=False)
    world = oracle_world(w)
    rng = np.random.default_rng(22)
    for i in _sample(w, inp, 3, 23):
        nr = _rotors(w, i)
        v = np.concatenate([x0[:, i], GAINS, inp.targets[:, i]]).astype(np.float64)
        L = _loss29(world, w, inp, i, x0, m0, goal, v)
        assert abs(loss[i] - L) <= 1e-4 * max(1.0, abs(L)), (i, loss[i], L)
        ds, dg, dt = rng.normal(size=13), rng.normal(size=12), rng.normal(size=4)
        _, jvp = O.vehicle_loss_jvp(world, nr, int(inp.modes[i]), v[25:29], inp.body[:, i].astype(np.float64),
                                    v[:13], m0[0:nr, i].astype(np.float64), GAINS, ds, dg, H_MODES,
                                    goal[:, i].astype(np.float64), W_POS, W_OMEGA, d_tgt4=dt)
        dot = float(gx[:, i].astype(np.float64) @ ds + gge[:, i].astype(np.float64) @ dg +
                    gt[:, i].astype(np.float64) @ dt)
        assert abs(dot - jvp) <= 1e-3 * max(1.0, abs(jvp)), (MODE_NAMES[int(inp.modes[i])], nr, i, dot, jvp)


def test_adjoint_every_mode_matches_fd_on_every_component():
    w = MODES_W
    inp = _mode_inputs(w, 31, gentle=True)
    x0, m0, goal, loss, sat, gx, gge, gt = _run_modes(w, inp, 31, gentle=True)
    # no clamp anywhere: every component is compared
    assert sat.sum() == 0, {MODE_NAMES[m]: int(sat[inp.modes == m].sum()) for m in MODE_NAMES}
    world = oracle_world(w)
    for i in _sample(w, inp, 2, 32):
        base = np.concatenate([x0[:, i], GAINS, inp.targets[:, i]]).astype(np.float64)
        g_fd = np.zeros(29)
        for k in range(29):
            h = 1e-6 * max(1.0, abs(base[k]))
            vp, vm = base.copy(), base.copy()
            vp[k] += h
            vm[k] -= h
            g_fd[k] = (_loss29(world, w, inp, i, x0, m0, goal, vp) - _loss29(world, w, inp, i, x0, m0, goal, vm)) / (2 * h)
        g_gpu = np.concatenate([gx[:, i], gge[:, i], gt[:, i]]).astype(np.float64)
        err = np.linalg.norm(g_gpu - g_fd) / max(np.linalg.norm(g_fd), 1e-6)
        assert err <= 1e-3, (MODE_NAMES[int(inp.modes[i])], _rotors(w, i), i, err, g_gpu, g_fd)
        # the target part alone (it is small next to the state part in some modes)
        et = np.linalg.norm(g_gpu[25:] - g_fd[25:]) / max(np.linalg.norm(g_fd[25:]), 1e-6)
        assert et <= 2e-3, (MODE_NAMES[int(inp.modes[i])], i, et, g_gpu[25:], g_fd[25:])


def test_autograd_target_gradient_matches_ag_backward():
    from paper_2305_16510_gb300.autograd import rollout_loss
    w = W.scaled(MODES_W, 512)
    inp = _mode_inputs(w, 41, gentle=False)
    x0, m0, goal, loss, sat, gx, gge, gt = _run_modes(w, inp, 41, gentle=False)
    fl = gpu_fleet(w, inp, 41)
    x0_t = torch.from_numpy(x0).cuda().requires_grad_(True)
    tg_t = torch.from_numpy(inp.targets).cuda().requires_grad_(True)
    gains_t = torch.tensor(GAINS, dtype=torch.float32, requires_grad=True)
    out = rollout_loss(fl, x0_t, gains_t, torch.from_numpy(m0).cuda(), H_MODES, torch.from_numpy(goal).cuda(),
                       W_POS, W_OMEGA, targets=tg_t)
    np.testing.assert_allclose(_np(out), loss, rtol=1e-6)
    out.sum().backward()
    np.testing.assert_allclose(_np(tg_t.grad), gt, rtol=1e-6, atol=1e-6 * np.abs(gt).max())
    np.testing.assert_allclose(_np(x0_t.grad), gx, rtol=1e-6, atol=1e-6 * np.abs(gx).max())
    fl.close()


def test_whole_horizon_tape_and_one_segment_tape_agree():
    """ag_rollout_loss keeps a tape of the whole horizon when it fits (the
    backward pass then recomputes every checkpoint segment in parallel), else
    one segment's tape (recomputed segment by segment in the sweep). A context
    whose hbm_budget_bytes leaves no room for the whole-horizon tape takes the
    second path. The two recompute the same steps in different kernels, where
    the compiler may contract multiply-adds differently, so they agree to
    float32 rounding (measured about 1e-6 relative), not bit for bit: each
    vehicle's gradient within 1e-4 relative, here over every mode and airframe
    with a horizon that is not a multiple of the checkpoint interval. The loss
    comes from the same record in both and is identical."""
    from paper_2305_16510_gb300.fleet import Fleet
    w = MODES_W
    inp = _mode_inputs(w, 41, gentle=False)
    horizon = 100                                   # segments of 32, 32, 32 and 4 steps
    n = w.n_envs
    full_tape_bytes = horizon * 21 * n * 4          # 25.8 MB
    outs = []
    for budget in (0, 12 << 20):                    # no limit; 12 MiB (the fleet, checkpoints, one segment)
        fl = Fleet(n, n_hexa=w.n_hexa, n_octo=w.n_octo, drag=w.drag, seed=41, hbm_budget_bytes=budget)
        fl.set_body(inp.body)
        fl.set_commands(inp.modes, inp.targets)
        fl.reset(None, 41)
        goal = torch.from_numpy(np.ascontiguousarray(inp.targets[0:3])).cuda()
        loss = torch.empty(n, dtype=torch.float32, device="cuda")
        gx = torch.empty((13, n), dtype=torch.float32, device="cuda")
        gg = torch.empty((12,), dtype=torch.float32, device="cuda")
        gge = torch.empty((12, n), dtype=torch.float32, device="cuda")
        gt = torch.empty((4, n), dtype=torch.float32, device="cuda")
        _abi.ag_rollout_loss(fl.ctx, horizon, W_POS, W_OMEGA, goal, loss)
        _abi.ag_backward(fl.ctx, None, gx, gg, gge, gt)
        torch.cuda.synchronize()
        outs.append([_np(t) for t in (loss, gx, gg, gge, gt)])
        fl.close()
    assert full_tape_bytes > 12 << 20
    full, seg = outs
    np.testing.assert_array_equal(full[0], seg[0])                     # loss
    for k in (1, 3, 4):                                                # per vehicle: x0, gains, targets
        diff = np.linalg.norm(full[k] - seg[k], axis=0)
        ref = np.maximum(np.linalg.norm(seg[k], axis=0), 1e-6)
        assert np.max(diff / ref) <= 1e-4, (k, np.max(diff / ref))
    assert np.linalg.norm(full[2] - seg[2]) <= 1e-4 * np.linalg.norm(seg[2])   # fleet gain sum
    assert np.abs(full[1]).max() > 0
