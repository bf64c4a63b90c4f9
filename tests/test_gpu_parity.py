"""CUDA path (through the C-ABI) against the FP64 oracle, element by element.

Tolerances: the FP32 state after 100 semi-implicit-Euler steps must match
the oracle within 1e-4 m in position and 1e-4 rad in attitude (the parity
bar of the fleet-step workload). Every other bound sits 5 to 15 times above
the error measured on its seeded case (each check records both when
AG_TOLERANCE_REPORT is set), and never above that bar except where noted:
one step from the same float32 state 2e-6 relative; rollouts of 60 to 100
steps 1e-5; the 1,000-step full-size rollout 1e-4 (position, relative to
1 + |p|) and 1e-4 rad.
Reset draws are compared bit for bit. Collision decisions whose squared
distance margin lies within 1e-5 m^2 of the radius are near-ties that float32
and float64 may decide differently; they are counted and excluded.
"""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import oracle as O
from harness import (attitude_error, box_margin, gpu_fleet, max_state_errors, oracle_fleet_from, oracle_world,
                     subset)
from paper_2305_16510_gb300 import _abi
from paper_2305_16510_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2305_16510_gb300 import build
    build.build()


def _np(t):
    return t.detach().cpu().numpy()


def _reset_pair(w, seed, inp=None):
    inp = inp or W.make_inputs(w, seed)
    fl = gpu_fleet(w, inp, seed)
    fl.reset(None, seed)
    orc = oracle_fleet_from(w, inp, np.zeros((13, w.n_envs)), np.zeros((8, w.n_envs)), np.zeros(w.n_envs, np.uint32),
                            seed)
    O.reset(oracle_world(w), orc, None, seed)
    return fl, orc, inp


# ------------------------------------------------------------------ resets --
def test_reset_draws_bit_exact_mixed_fleet():
    w = W.scaled(W.WORKLOADS["mixed"], 1000)
    fl, orc, inp = _reset_pair(w, 2024)
    st = _np(fl.state())
    np.testing.assert_array_equal(st, orc.state.astype(np.float32))
    mot = _np(fl.motors())
    np.testing.assert_array_equal(mot, orc.motors.astype(np.float32))
    np.testing.assert_array_equal(_np(fl.epoch()).astype(np.uint32), orc.epoch)
    col, ids = fl.events()
    assert sorted(_np(ids).tolist()) == list(range(w.n_envs))
    assert int(_np(col).sum()) == 0
    # a masked reset with another seed
    mask = W.reset_mask(w.n_envs, 0.3, np.random.default_rng(5))
    fl.reset(mask, 99)
    O.reset(oracle_world(w), orc, mask, 99)
    np.testing.assert_array_equal(_np(fl.state()), orc.state.astype(np.float32))
    np.testing.assert_array_equal(_np(fl.motors()), orc.motors.astype(np.float32))
    np.testing.assert_array_equal(_np(fl.epoch()).astype(np.uint32), orc.epoch)
    _, ids = fl.events()
    assert sorted(_np(ids).tolist()) == np.flatnonzero(mask).tolist()
    fl.close()


def test_reset_draws_bit_exact_one_million():
    w = W.WORKLOADS["obstacles"]
    n = w.n_envs
    inp = W.Inputs(np.zeros(n, np.uint8), np.zeros((4, n), np.float32), W.body(w, np.random.default_rng(0)), None)
    w0 = W.Workload(**{**w.__dict__, "n_obstacles": 0})
    fl = gpu_fleet(w0, inp, 7)
    fl.reset(None, 0x1234_5678_9ABC_DEF0)
    fl.reset(W.reset_mask(n, 0.5, np.random.default_rng(1)), 0x1234_5678_9ABC_DEF0)
    orc = oracle_fleet_from(w0, inp, np.zeros((13, n)), np.zeros((8, n)), np.zeros(n, np.uint32), 0)
    O.reset(oracle_world(w0), orc, None, 0x1234_5678_9ABC_DEF0)
    O.reset(oracle_world(w0), orc, W.reset_mask(n, 0.5, np.random.default_rng(1)), 0x1234_5678_9ABC_DEF0)
    np.testing.assert_array_equal(_np(fl.state()), orc.state.astype(np.float32))
    fl.close()


# ---------------------------------------------------------- full rollouts --
def test_parity_position_mode_1024_quads_100_steps(within_tolerance):
    w = W.WORKLOADS["parity"]
    fl, orc, _ = _reset_pair(w, 1)
    fl.step(100)
    O.rollout(oracle_world(w), orc, 100, n_threads=8)
    dp, dv, dang, dw = max_state_errors(_np(fl.state()), orc.state)
    # T1: the parity bar of the 1,024-quad, 100-step workload
    within_tolerance("position [m]", dp.max(), 1e-4)
    within_tolerance("attitude [rad]", dang.max(), 1e-4)
    within_tolerance("velocity [m/s]", dv.max(), 5e-5)
    within_tolerance("body rate [rad/s]", dw.max(), 3e-4)
    # the oracle's controller really moved the fleet towards its targets
    assert np.mean(np.abs(orc.state[0:3] - orc.targets[0:3])) < 2.0


@pytest.mark.parametrize("mode_mix,integ,sub", [
    ((W.MODE_POSITION,), 1, 4),
    ((W.MODE_BODY_VEL,), 0, 1),
    ((W.MODE_BODY_VEL,), 1, 4),
    ((W.MODE_ATT_THRUST,), 0, 1),
    ((W.MODE_ATT_THRUST,), 1, 2),
    ((W.MODE_POSITION, W.MODE_BODY_VEL, W.MODE_ATT_THRUST), 1, 4),
])
def test_parity_each_mode_and_integrator(mode_mix, integ, sub, within_tolerance):
    # 1,000 envs: several 128-thread blocks and a ragged last block
    w = W.Workload("modes", 1000, sub, integ, 0, 1000, 0, 0, mode_mix=mode_mix)
    fl, orc, _ = _reset_pair(w, 11)
    fl.step(100)
    O.rollout(oracle_world(w), orc, 100, n_threads=8)
    dp, dv, dang, dw = max_state_errors(_np(fl.state()), orc.state)
    scale = 1.0 + np.max(np.abs(orc.state[0:3]), axis=0)
    # T2
    within_tolerance("position / (1 + |p|) [m]", np.max(dp / scale), 1e-5)
    within_tolerance("attitude [rad]", dang.max(), 5e-5)


def test_parity_mixed_rotor_types_drag_and_random_bodies(within_tolerance):
    w = W.scaled(W.WORKLOADS["mixed"], 2000)
    fl, orc, _ = _reset_pair(w, 3)
    fl.step(60)
    O.rollout(oracle_world(w), orc, 60, n_threads=8)
    dp, dv, dang, dw = max_state_errors(_np(fl.state()), orc.state)
    # T3
    within_tolerance("position [m]", dp.max(), 1e-5)
    within_tolerance("attitude [rad]", dang.max(), 1e-5)
    mot = _np(fl.motors())
    within_tolerance("motor thrust [N]", np.max(np.abs(mot - orc.motors)), 1e-5)


def test_wrench_mode_free_fall_and_hover_fixed_point():
    n = 300
    w = W.Workload("wrench", n, 1, 0, 0, n, 0, 0, mode_mix=(W.MODE_WRENCH,))
    fl, orc, inp = _reset_pair(w, 5)
    # zero commanded wrench: the motors spin down through the lag, then free fall
    fl.step(50)
    O.rollout(oracle_world(w), orc, 50)
    np.testing.assert_allclose(_np(fl.state())[0:3], orc.state[0:3], atol=1e-4)
    # hover: at the position target, level at the yaw target, at rest
    tg = np.zeros((4, n), np.float32)
    tg[0:3] = np.random.default_rng(1).uniform(-1, 1, (3, n))
    st = np.zeros((13, n), np.float32)
    st[0:3] = tg[0:3]
    st[6] = 1.0
    mot = np.zeros((8, n), np.float32)
    mot[0:4] = np.float32(0.75 * 9.81 / 4)
    fl.set_commands(np.zeros(n, np.uint8), tg)
    fl.set_state(st, mot)
    fl.step(100)
    np.testing.assert_allclose(_np(fl.state()), st, atol=2e-5)
    fl.close()


def test_torque_free_rk4_conserves_momentum_and_energy_and_falls_on_the_parabola():
    """Pinned by the physics, not the oracle: with zero wrench and an
    asymmetric inertia the world angular momentum R J Omega and the kinetic
    energy 1/2 Omega^T J Omega are invariants, and the centre of mass follows
    p0 + v0 t - 1/2 g t^2 e3, which RK4 integrates exactly. 1,000 steps of
    4 RK4 substeps in float32."""
    from paper_2305_16510_gb300.fleet import Fleet
    n, steps, dt = 512, 1000, 0.01
    rng = np.random.default_rng(77)
    fl = Fleet(n, substeps_per_step=4, integrator=_abi.AG_INTEG_RK4, motor_tau=0.0)
    J = np.array([0.007, 0.009, 0.012])
    fl.set_body(np.tile(np.array([[0.75], [J[0]], [J[1]], [J[2]]], np.float32), (1, n)))
    fl.set_commands(np.full(n, W.MODE_WRENCH, np.uint8), np.zeros((4, n), np.float32))
    st = np.zeros((13, n), np.float32)
    st[0:3] = rng.uniform(-2, 2, (3, n))
    st[3:6] = rng.normal(0, 1.0, (3, n))
    q = rng.normal(size=(4, n))
    st[6:10] = q / np.linalg.norm(q, axis=0)
    st[10:13] = rng.normal(0, 1.5, (3, n))
    fl.set_state(st, np.zeros((8, n), np.float32))

    def invariants(s):
        s = s.astype(np.float64)
        R = Rotation.from_quat(np.stack([s[7], s[8], s[9], s[6]], axis=1)).as_matrix()
        Jw = J[:, None] * s[10:13]
        return np.einsum("nij,jn->in", R, Jw), 0.5 * np.sum(s[10:13] * Jw, axis=0)

    L0, E0 = invariants(st)
    fl.step(steps)
    s1 = _np(fl.state())
    L1, E1 = invariants(s1)
    # float32 rounding over 4,000 substeps; a modelling error (a dropped gyroscopic term, a wrong
    # sign) misses these by orders of magnitude
    assert np.all(np.linalg.norm(L1 - L0, axis=0) <= 5e-4 * np.linalg.norm(L0, axis=0))
    assert np.all(np.abs(E1 - E0) <= 5e-4 * E0)
    np.testing.assert_allclose(np.linalg.norm(s1[6:10].astype(np.float64), axis=0), 1.0, atol=1e-6)
    t = steps * dt
    p_exact = st[0:3].astype(np.float64) + st[3:6].astype(np.float64) * t
    p_exact[2] -= 0.5 * 9.81 * t * t
    v_exact = st[3:6].astype(np.float64)
    v_exact[2] -= 9.81 * t
    # |p| reaches ~500 m: 4,000 float32 additions at that size round to ~2e-4 of it
    assert np.all(np.abs(s1[0:3] - p_exact) <= 2e-4 * (1 + np.abs(p_exact)))
    assert np.all(np.abs(s1[3:6] - v_exact) <= 2e-4 * (1 + np.abs(v_exact)))
    fl.close()


def test_yaw_torque_spins_a_level_hover_with_constant_angular_acceleration():
    """Pinned by the physics: a level vehicle commanded f = m g and a small
    yaw moment M_z (wrench mode, no motor lag) keeps its position and turns
    about +z with psi(t) = psi0 + w0 t + 1/2 (M_z / J_z) t^2, on quad, hexa and
    octo airframes. Bounds: with A and its pseudo-inverse rounded to float32,
    A A^+ - I is ~1e-7, so the 7.4 N thrust leaks ~7e-7 N m into each moment.
    Open loop over 2 s that is ~1e-4 rad/s of yaw rate, ~1e-4 of tilt and
    ~1e-3 m of drift; the bounds below sit ~10x above. A wrong torque sign or
    scale misses them by orders of magnitude."""
    from paper_2305_16510_gb300.fleet import Fleet
    n_q, n_h, n_o = 256, 256, 256
    n = n_q + n_h + n_o
    rng = np.random.default_rng(21)
    fl = Fleet(n, n_hexa=n_h, n_octo=n_o, substeps_per_step=4, integrator=_abi.AG_INTEG_RK4, motor_tau=0.0)
    m, jz = 0.75, 0.012
    psi0 = rng.uniform(-1, 1, n)
    w0 = rng.uniform(-1, 1, n)
    mz = rng.uniform(-2e-3, 2e-3, n)
    tg = np.zeros((4, n), np.float32)
    tg[0] = m * 9.81
    tg[3] = mz
    fl.set_commands(np.full(n, W.MODE_WRENCH, np.uint8), tg)
    st = np.zeros((13, n), np.float32)
    st[0:3] = rng.uniform(-2, 2, (3, n))
    st[6], st[9] = np.cos(psi0 / 2), np.sin(psi0 / 2)
    st[12] = w0
    fl.set_state(st, np.zeros((8, n), np.float32))
    steps = 200                                      # 2 s
    fl.step(steps)
    s1 = _np(fl.state()).astype(np.float64)
    t = steps * 0.01
    alpha = tg[3].astype(np.float64) / jz
    psi = 2 * np.arctan2(s1[9], s1[6])
    want = psi0 + w0 * t + 0.5 * alpha * t * t
    err = np.angle(np.exp(1j * (psi - want)))       # wrapped to (-pi, pi]
    assert np.max(np.abs(err)) < 1e-4, np.max(np.abs(err))
    np.testing.assert_allclose(s1[12], w0 + alpha * t, atol=1e-3)
    np.testing.assert_allclose(s1[7:9], 0.0, atol=1e-3)             # stays level
    np.testing.assert_allclose(s1[0:3], st[0:3], atol=1e-2)         # hovers in place
    fl.close()


def test_position_control_converges_from_small_errors_on_every_airframe():
    """Pinned by the control law's stability (Lee et al. 2011, the position
    controller of Sec. I): from 0.1 m and 5 deg off a hover setpoint, quad,
    hexa and octo fleets settle within 1e-3 m and 1e-3 (|e_R|) in 10 s."""
    from paper_2305_16510_gb300.fleet import Fleet
    n_q, n_h, n_o = 2048, 1024, 1024
    n = n_q + n_h + n_o
    rng = np.random.default_rng(12)
    fl = Fleet(n, n_hexa=n_h, n_octo=n_o)
    pd = rng.uniform(-3, 3, (3, n))
    psi_d = rng.uniform(-3, 3, n)
    e = rng.normal(size=(3, n))
    e *= 0.1 / np.linalg.norm(e, axis=0)
    ax = rng.normal(size=(n, 3))
    ax /= np.linalg.norm(ax, axis=1, keepdims=True)
    R0 = Rotation.from_euler("Z", psi_d[:, None]) * Rotation.from_rotvec(np.radians(5) * ax)
    q = R0.as_quat()                              # x, y, z, w
    st = np.zeros((13, n), np.float32)
    st[0:3] = pd + e
    st[6], st[7], st[8], st[9] = q[:, 3], q[:, 0], q[:, 1], q[:, 2]
    mot = np.zeros((8, n), np.float32)
    n_rot = np.array([4] * n_q + [6] * n_h + [8] * n_o)
    for k in range(8):
        mot[k] = np.where(k < n_rot, 0.75 * 9.81 / n_rot, 0.0)
    tg = np.vstack([pd, psi_d[None]]).astype(np.float32)
    fl.set_commands(np.zeros(n, np.uint8), tg)
    fl.set_state(st, mot)
    fl.step(1000)
    s1 = _np(fl.state()).astype(np.float64)
    assert np.max(np.linalg.norm(s1[0:3] - pd, axis=0)) < 1e-3
    R = Rotation.from_quat(np.stack([s1[7], s1[8], s1[9], s1[6]], axis=1)).as_matrix()
    Rd = Rotation.from_euler("Z", psi_d[:, None]).as_matrix()
    E = np.einsum("nji,njk->nik", Rd, R) - np.einsum("nji,njk->nik", R, Rd)
    eR = 0.5 * np.stack([E[:, 2, 1], E[:, 0, 2], E[:, 1, 0]], axis=1)
    assert np.max(np.linalg.norm(eR, axis=1)) < 1e-3
    fl.close()


# -------------------------------------------------------------- obstacles --
def _teacher_forced_steps(w, seed, n_calls, within_tolerance, plain=False):
    """One step per call; after each call the oracle advances the GPU's
    pre-call state by one step and the two are compared."""
    fl, _, inp = _reset_pair(w, seed)
    world = oracle_world(w)
    world_free = oracle_world(W.Workload(**{**w.__dict__, "n_obstacles": 0}))
    n_ambiguous = n_hits = 0
    worst_p = worst_ang = 0.0
    for _ in range(n_calls):
        s0, m0, e0 = _np(fl.state()), _np(fl.motors()), _np(fl.epoch()).astype(np.uint32)
        (fl.step_plain if plain else fl.step)(1)
        s1, col, ids = _np(fl.state()), *[_np(x) for x in fl.events()]
        # oracle: the same step from the same float32 state
        pre = oracle_fleet_from(w, inp, s0, m0, e0, seed)
        pre.boxes = None
        O.rollout(world_free, pre, 1)
        amb = np.abs(box_margin(pre.state[0:3], inp.boxes.astype(np.float64))) < 1e-5
        orc = oracle_fleet_from(w, inp, s0, m0, e0, seed)
        ocol, _ = O.rollout(world, orc, 1)
        ok = ~amb
        n_ambiguous += int(amb.sum())
        n_hits += int(ocol[ok].sum())
        np.testing.assert_array_equal(col[ok], ocol[ok])
        assert set(ids.tolist()) == set(np.flatnonzero(col).tolist())
        hit = ok & (ocol == 1)
        # a reset env holds its Philox draw bit for bit
        np.testing.assert_array_equal(s1[:, hit], orc.state[:, hit].astype(np.float32))
        free = ok & (ocol == 0)
        dp, dv, dang, dw = max_state_errors(s1[:, free], orc.state[:, free])
        scale = 1.0 + np.max(np.abs(orc.state[0:3, free]), axis=0)
        worst_p = max(worst_p, float(np.max(dp / scale)))
        worst_ang = max(worst_ang, float(dang.max()))
    # T4: one step from the same float32 state
    within_tolerance("position / (1 + |p|) per step [m]", worst_p, 2e-6)
    within_tolerance("attitude per step [rad]", worst_ang, 2e-6)
    return n_hits, n_ambiguous


def test_obstacle_collisions_and_resets_teacher_forced(within_tolerance):
    w = W.scaled(W.WORKLOADS["obstacles"], 2048)
    hits, amb = _teacher_forced_steps(w, 21, 25, within_tolerance)
    assert hits > 20           # the workload does collide
    within_tolerance("near-tie env-steps excluded (of 51,200)", amb, 5)


def test_plain_path_matches_oracle_teacher_forced(within_tolerance):
    w = W.scaled(W.WORKLOADS["obstacles"], 1000)
    hits, amb = _teacher_forced_steps(w, 22, 10, within_tolerance, plain=True)
    assert hits > 5
    within_tolerance("near-tie env-steps excluded (of 10,000)", amb, 5)


def _allclose_ratio(a, b, atol, rtol):
    """max |a - b| / (atol + rtol |b|): at most 1 where assert_allclose passes."""
    a64, b64 = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.max(np.abs(a64 - b64) / (atol + rtol * np.abs(b64)))) if a64.size else 0.0


def test_plain_and_fused_agree(within_tolerance):
    w = W.scaled(W.WORKLOADS["obstacles"], 3000)
    inp = W.make_inputs(w, 8)
    a, b = gpu_fleet(w, inp, 8), gpu_fleet(w, inp, 8)
    a.reset(None, 8)
    b.reset(None, 8)
    a.step(20)
    b.step_plain(20)
    sa, sb = _np(a.state()), _np(b.state())
    ca, ia = a.events()
    cb, ib = b.events()
    same = (_np(ca) == _np(cb)) & (_np(a.epoch()) == _np(b.epoch()))
    # T5: rare float32 near-ties may differ between the two evaluation orders
    within_tolerance("fraction of envs whose collisions differ", 1.0 - same.mean(), 0.002)
    within_tolerance("|fused - plain| / (1e-5 + 1e-6 |x|)", _allclose_ratio(sa[:, same], sb[:, same], 1e-5, 1e-6), 1.0)
    a.close()
    b.close()


def test_per_mode_loops_equal_the_branching_loop(monkeypatch):
    """In the grouped thread order a warp of one command mode runs the step
    loop compiled for that mode; in the identity order every warp runs the
    branching loop. Every fused multiply-add of the step is explicit and
    nothing else is contracted, so the two must agree bit for bit: a mixed
    fleet (all four command modes, quads, RK4, 16 boxes, collisions and
    resets) stepped 200 steps in one call, in both orders."""
    w = W.Workload("modes", 6000, 4, 1, 16, 6000, 0, 0,
                   mode_mix=(W.MODE_POSITION, W.MODE_BODY_VEL, W.MODE_ATT_THRUST, W.MODE_WRENCH))
    inp = W.make_inputs(w, 31)
    out = []
    for order in ("grouped", "identity"):
        if order == "identity":
            monkeypatch.setenv("AG_FUSED_ORDER", "identity")
        fl = gpu_fleet(w, inp, 31)
        fl.reset(None, 31)
        fl.step(200)
        col, ids = fl.events()
        out.append((_np(fl.state()), _np(fl.motors()), _np(fl.epoch()), _np(col), np.sort(_np(ids))))
        fl.close()
    monkeypatch.delenv("AG_FUSED_ORDER")
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)
    assert (out[0][2].astype(np.int64) > 1).sum() > 10        # collision resets happened


def test_skipped_collision_tests_change_no_decision(monkeypatch):
    """The fused step skips a vehicle's collision test while the distance it
    has moved since its last exact test stays below that test's clearance
    (minus a rounding slack). AG_FUSED_SKIP=0 runs the exact test at every
    step instead; both runs must agree bit for bit. The boxes are packed
    closer than in the bench recipe (centres U[-2.5, 2.5]^3) so that vehicles
    pass near them often, and one call runs 300 steps so the skip is in
    force for long stretches."""
    w = W.scaled(W.WORKLOADS["obstacles"], 8192)
    inp = W.make_inputs(w, 44)
    boxes = inp.boxes.copy()
    boxes[:, 0:3] = np.random.default_rng(45).uniform(-2.5, 2.5, (w.n_obstacles, 3, w.n_envs)).astype(np.float32)
    inp = W.Inputs(inp.modes, inp.targets, inp.body, boxes)
    out, tests = [], []
    for skip in ("1", "0"):
        monkeypatch.setenv("AG_FUSED_SKIP", skip)
        fl = gpu_fleet(w, inp, 44)
        fl.reset(None, 44)
        fl.step(300)
        col, ids = fl.events()
        out.append((_np(fl.state()), _np(fl.motors()), _np(fl.epoch()), _np(col), np.sort(_np(ids))))
        tests.append(_abi.ag_collision_tests_run(fl.ctx))
        fl.close()
    monkeypatch.delenv("AG_FUSED_SKIP")
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)
    # the exact run tests every environment after every step; the default run skips most tests
    assert tests[1] == w.n_envs * 300
    assert 0 < tests[0] < 0.8 * tests[1]
    assert (out[0][2].astype(np.int64) - 1).sum() > 500   # hundreds of collision resets after the first draw
    assert out[0][3].mean() > 0.02


def test_max_obstacles_and_single_env():
    for n, n_obs in ((1, 3), (77, 64)):
        w = W.Workload("maxobs", n, 2, 1, n_obs, n, 0, 0, mode_mix=(W.MODE_POSITION, W.MODE_ATT_THRUST))
        inp = W.make_inputs(w, 4)
        fl = gpu_fleet(w, inp, 4)
        fl.reset(None, 4)
        s0, m0, e0 = _np(fl.state()), _np(fl.motors()), _np(fl.epoch()).astype(np.uint32)
        fl.step(1)
        orc = oracle_fleet_from(w, inp, s0, m0, e0, 4)
        ocol, _ = O.rollout(oracle_world(w), orc, 1)
        col, _ = fl.events()
        np.testing.assert_array_equal(_np(col), ocol)
        s1 = _np(fl.state())
        dp, _, dang, _ = max_state_errors(s1, orc.state)
        assert dp.max() <= 2e-5 and dang.max() <= 2e-5
        fl.close()


# --------------------------------------------- launch configuration checks --
def test_one_call_of_many_steps_equals_single_step_calls(within_tolerance):
    w = W.scaled(W.WORKLOADS["obstacles"], 1500)
    inp = W.make_inputs(w, 31)
    a, b = gpu_fleet(w, inp, 31), gpu_fleet(w, inp, 31)
    a.reset(None, 31)
    b.reset(None, 31)
    a.step(12)
    for _ in range(12):
        b.step(1)
    same = _np(a.epoch()) == _np(b.epoch())
    # T6
    within_tolerance("fraction of envs whose resets differ", 1.0 - same.mean(), 0.002)
    within_tolerance("|one call - 12 calls| / (1e-5 + 1e-6 |x|)",
                     _allclose_ratio(_np(a.state())[:, same], _np(b.state())[:, same], 1e-5, 1e-6), 1.0)
    a.close()
    b.close()


def test_fused_steps_captured_in_a_cuda_graph_replay_bit_exactly():
    """ag_step issues its launches on the context's stream without allocating
    or synchronising, so a loop of calls can be captured in a CUDA graph: 5
    captured calls replayed 3 times equal 15 direct calls bit for bit,
    collision resets included."""
    from paper_2305_16510_gb300.fleet import Fleet
    w = W.Workload("graph", 3000, 4, 1, 8, 3000, 0, 0)
    inp = W.make_inputs(w, 6)
    results = []
    for use_graph in (False, True):
        side = torch.cuda.Stream()          # capture needs a stream other than the legacy default one
        with torch.cuda.stream(side):
            fl = Fleet(w.n_envs, substeps_per_step=4, integrator=1, n_obstacles=8, seed=6, stream=side)
            fl.set_body(inp.body)
            fl.set_commands(inp.modes, inp.targets)
            fl.set_obstacles(inp.boxes)
            fl.reset(None, 6)
            fl.step(1)                      # first use of the kernel outside the capture
            hits = torch.zeros(w.n_envs, dtype=torch.int32, device=fl.device)
            col = torch.empty(w.n_envs, dtype=torch.uint8, device=fl.device)
        torch.cuda.synchronize()

        def calls():
            for _ in range(5):
                _abi.ag_step(fl.ctx, 4)
                _abi.ag_get_state(fl.ctx, collided=col)
                hits.add_(col)

        if use_graph:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=side):
                calls()
            for _ in range(3):
                g.replay()
        else:
            with torch.cuda.stream(side):
                for _ in range(3):
                    calls()
        torch.cuda.synchronize()
        results.append((_np(fl.state()), _np(fl.motors()), _np(fl.epoch()), _np(hits)))
        fl.close()
    for a, b in zip(*results):
        np.testing.assert_array_equal(a, b)
    assert results[0][3].sum() > 0                 # collisions (and resets) happened in the 15 calls


def test_checkpoint_resume_is_bit_exact():
    w = W.scaled(W.WORKLOADS["obstacles"], 700)
    inp = W.make_inputs(w, 12)
    fl = gpu_fleet(w, inp, 12)
    fl.reset(None, 12)
    fl.step(5)
    ck = (fl.state().clone(), fl.motors().clone(), fl.epoch().clone())
    fl.step(10)
    s1, e1 = _np(fl.state()), _np(fl.epoch())
    fl.set_state(*ck)
    fl.step(10)
    np.testing.assert_array_equal(_np(fl.state()), s1)
    np.testing.assert_array_equal(_np(fl.epoch()), e1)
    fl.close()


def test_host_buffers_round_trip_through_the_abi():
    w = W.WORKLOADS["parity"]
    inp = W.make_inputs(w, 2)
    fl = gpu_fleet(w, inp, 2)
    fl.reset(None, 2)
    host = np.empty((13, w.n_envs), np.float32)
    _abi.ag_get_state(fl.ctx, state=host)
    fl.synchronize()
    np.testing.assert_array_equal(host, _np(fl.state()))
    host[0] += 1.0
    _abi.ag_set_state(fl.ctx, host)
    np.testing.assert_array_equal(_np(fl.state()), host)
    fl.close()


def test_invalid_arguments_leave_context_usable():
    w = W.Workload("inv", 64, 4, 1, 0, 64, 0, 0)
    inp = W.make_inputs(w, 1)
    fl = gpu_fleet(w, inp, 1)
    with pytest.raises(_abi.AgError) as e:
        _abi.ag_step(fl.ctx, 3)
    assert e.value.status == _abi.AG_ERR_INVALID
    with pytest.raises(_abi.AgError):
        _abi.ag_step(fl.ctx, 0)
    # step counts that do not fit the kernels' int step counter
    from paper_2305_16510_gb300.fleet import Fleet
    one = Fleet(64)
    for n_sub in (1 << 31, (1 << 32) - 1):
        with pytest.raises(_abi.AgError) as e:
            _abi.ag_step(one.ctx, n_sub)
        assert e.value.status == _abi.AG_ERR_INVALID
    goal, loss = torch.zeros((3, 64), device=one.device), torch.empty(64, device=one.device)
    with pytest.raises(_abi.AgError) as e:
        _abi.ag_rollout_loss(one.ctx, (1 << 30) + 1, 1.0, 0.01, goal, loss)
    assert e.value.status == _abi.AG_ERR_INVALID
    one.step(1)
    assert np.isfinite(_np(one.state())).all()
    one.close()
    fl.reset(None, 1)
    fl.step(2)
    assert np.isfinite(_np(fl.state())).all()
    cfg = _abi.ag_config_default()
    cfg.n_envs = 1 << 20
    cfg.n_quad = 1 << 20
    cfg.hbm_budget_bytes = 1 << 20
    with pytest.raises(_abi.AgError) as e:
        _abi.ag_create(cfg, torch.cuda.current_stream().cuda_stream)
    assert e.value.status == _abi.AG_ERR_OOM
    fl.close()


# ----------------------------------------- full size, sampled, bench launch --
def test_full_size_obstacle_fleet_sampled_against_oracle(within_tolerance):
    """1,048,576 quads, 16 boxes each, one ag_step of 1,000 steps (the launch
    the bench times); 384 sampled envs are re-simulated by the oracle step by
    step from the same initial draw, near-tie envs excluded."""
    w = W.WORKLOADS["obstacles"]
    seed = 1
    inp = W.make_inputs(w, seed)
    fl = gpu_fleet(w, inp, seed)
    fl.reset(None, seed)
    s0, m0, e0 = _np(fl.state()), _np(fl.motors()), _np(fl.epoch()).astype(np.uint32)
    fl.step(1000)
    s1 = _np(fl.state())
    col = _np(fl.events()[0])
    e1 = _np(fl.epoch()).astype(np.uint32)
    fl.close()
    idx = np.sort(np.random.default_rng(0).choice(w.n_envs, 384, replace=False))
    ws, ins = subset(w, inp, idx)
    boxes = ins.boxes.astype(np.float64)
    world, world_free = oracle_world(ws), oracle_world(W.Workload(**{**ws.__dict__, "n_obstacles": 0}))
    orc = oracle_fleet_from(ws, ins, s0[:, idx], m0[:, idx], e0[idx], seed)
    ok = np.ones(len(idx), bool)
    any_hit = np.zeros(len(idx), np.uint8)
    for _ in range(1000):
        # near-tie check on the pre-collision position of this step
        pre = oracle_fleet_from(ws, ins, orc.state, orc.motors, orc.epoch, seed)
        pre.boxes = None
        O.rollout(world_free, pre, 1)
        ok &= np.abs(box_margin(pre.state[0:3], boxes)) >= 1e-5
        c, _ = O.rollout(world, orc, 1, env_ids=idx)    # resets draw with the global env id
        any_hit |= c
    # T7
    within_tolerance("fraction of sampled envs with a near-tie step", 1.0 - ok.mean(), 0.01)
    np.testing.assert_array_equal(e1[idx][ok], orc.epoch[ok])
    np.testing.assert_array_equal(col[idx][ok], any_hit[ok])
    dp, dv, dang, dw = max_state_errors(s1[:, idx[ok]], orc.state[:, ok])
    scale = 1.0 + np.max(np.abs(orc.state[0:3, ok]), axis=0)
    within_tolerance("position / (1 + |p|) after 1,000 steps [m]", np.max(dp / scale), 1e-4)
    within_tolerance("attitude after 1,000 steps [rad]", dang.max(), 1e-4)


def test_full_size_mixed_fleet_with_reset_masks_sampled_against_oracle(within_tolerance):
    """4,194,304 vehicles (40 % quad, 40 % hexa, 20 % octo), randomised mass and
    inertia, drag, body-velocity commands: the workload's 500 steps in calls of
    50 with a 1 % Bernoulli reset mask after each call. The reset words are
    compared bit for bit; 384 sampled envs are re-simulated by the oracle."""
    w = W.WORKLOADS["mixed"]
    seed = 4
    inp = W.make_inputs(w, seed)
    fl = gpu_fleet(w, inp, seed)
    fl.reset(None, seed)
    s0, m0, e0 = _np(fl.state()), _np(fl.motors()), _np(fl.epoch()).astype(np.uint32)
    idx = np.sort(np.random.default_rng(5).choice(w.n_envs, 384, replace=False))
    ws, ins = subset(w, inp, idx)
    assert ws.n_quad > 0 and ws.n_hexa > 0 and ws.n_octo > 0
    orc = oracle_fleet_from(ws, ins, s0[:, idx], m0[:, idx], e0[idx], seed)
    world = oracle_world(ws)
    rng = np.random.default_rng(6)
    for call in range(10):
        fl.step(50)
        O.rollout(world, orc, 50)
        mask = W.reset_mask(w.n_envs, 0.01, rng)
        pre = _np(fl.state())
        fl.reset(mask, seed + call + 1)
        post = _np(fl.state())
        hit = mask.astype(bool)
        # untouched envs keep their state; reset envs hold their Philox draw
        np.testing.assert_array_equal(post[:, ~hit], pre[:, ~hit])
        ids = np.flatnonzero(hit)[:2000]
        ep = _np(fl.epoch()).astype(np.uint32)
        for i in ids[:200]:
            d = O.sample_reset(seed + call + 1, int(i), int(ep[i]))
            np.testing.assert_array_equal(post[0:10, i], d)
            assert np.all(post[10:13, i] == 0.0)
        O.reset(world, orc, mask[idx], seed + call + 1, env_ids=idx)
    s1 = _np(fl.state())
    mot = _np(fl.motors())
    fl.close()
    dp, dv, dang, dw = max_state_errors(s1[:, idx], orc.state)
    # T8
    within_tolerance("position [m]", dp.max(), 1e-4)
    within_tolerance("attitude [rad]", dang.max(), 3e-5)
    within_tolerance("motor thrust [N]", np.max(np.abs(mot[:, idx] - orc.motors)), 1e-5)


def test_injected_failure_is_sticky_and_the_context_still_destroys():
    """A failure injected on the host behaves as a CUDA error does: every later
    call but ag_last_error and ag_destroy returns AG_ERR_STATE, the message is
    kept, and the device is never touched by the failure itself."""
    from paper_2305_16510_gb300.fleet import Fleet
    fl = Fleet(256)
    fl.reset(None, 1)
    _abi.ag_inject_failure(fl.ctx, "link to the flight computer lost")
    for call in (lambda: fl.step(1), lambda: fl.state(), lambda: fl.reset(None, 2),
                 lambda: _abi.ag_set_commands(fl.ctx, None, None)):
        with pytest.raises(_abi.AgError) as e:
            call()
        assert e.value.status == _abi.AG_ERR_STATE
    assert _abi.ag_last_error(fl.ctx) == "link to the flight computer lost"
    fl.close()
    # a fresh context on the same device works
    fl2 = Fleet(256)
    fl2.reset(None, 1)
    fl2.step(2)
    assert np.isfinite(_np(fl2.state())).all()
    fl2.close()


def test_setters_reject_broken_bodies_and_boxes_and_keep_the_context():
    """ag_set_body and ag_set_obstacles check their documented preconditions
    (finite positive masses and inertias; finite centres, positive
    half-extents, unit quaternions) on host and device arrays before anything
    is copied, so a rejected call leaves the context as it was."""
    w = W.Workload("checks", 300, 1, 0, 4, 300, 0, 0)
    inp = W.make_inputs(w, 2)
    fl = gpu_fleet(w, inp, 2)
    fl.reset(None, 2)
    boxes0 = _np(fl.obstacles()).copy()
    bodies = []
    for r, v in ((0, 0.0), (2, -0.01), (3, np.nan), (1, np.inf)):
        b = inp.body.copy()
        b[r, 17] = v
        bodies.append(b)
    boxes = []
    for k, f, v in ((0, 4, 0.0), (1, 0, np.nan), (2, 3, -0.5)):
        b = boxes0.copy()
        b[k, f, 5] = v
        boxes.append(b)
    b = boxes0.copy()
    b[3, 6:10, 9] *= 1.01               # not a unit quaternion
    boxes.append(b)
    for arr, setter in [(x, _abi.ag_set_body) for x in bodies] + [(x, _abi.ag_set_obstacles) for x in boxes]:
        for where in ("host", "device"):
            src = np.ascontiguousarray(arr) if where == "host" else torch.from_numpy(np.ascontiguousarray(arr)).cuda()
            with pytest.raises(_abi.AgError) as e:
                setter(fl.ctx, src)
            assert e.value.status == _abi.AG_ERR_INVALID, (setter.__name__, where)
    np.testing.assert_array_equal(_np(fl.obstacles()), boxes0)
    # still usable, and the body is the one set before
    fl.step(5)
    st = _np(fl.state())
    assert np.isfinite(st).all()
    ref = gpu_fleet(w, inp, 2)
    ref.reset(None, 2)
    ref.step(5)
    np.testing.assert_array_equal(_np(ref.state()), st)
    ref.close()
    fl.close()
