"""Pins of the FP64 oracle against what the paper and the mathematics fix.

No GPU. Each test checks the oracle against something other than itself: a
closed form, an invariant of the physics, an independent library routine
(scipy rotations, numpy cross products), brute force on tiny inputs, or
published known-answer vectors. Each is chosen so that a plausible mistake in
the oracle (a dropped term, a flipped sign, a transposed operand, a wrong
index or coefficient) makes at least one of them fail.
"""
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle as O

G = 9.81
BODY = np.array([0.75, 0.007, 0.007, 0.012])
GAINS = np.array([2, 2, 3, 2, 2, 2, 1.2, 1.2, 0.6, 0.2, 0.2, 0.1], dtype=np.float64)
HERE = os.path.dirname(os.path.abspath(__file__))


def quat_wxyz(rot: Rotation) -> np.ndarray:
    x, y, z, w = rot.as_quat()
    return np.array([w, x, y, z])


def state13(p=(0, 0, 0), v=(0, 0, 0), q=(1, 0, 0, 0), w=(0, 0, 0)):
    return np.array(list(p) + list(v) + list(q) + list(w), dtype=np.float64)


# ------------------------------------------------------------ hat / vee / R --
def test_hat_vee_identities():
    rng = np.random.default_rng(1)
    for _ in range(20):
        a, b = rng.normal(size=3), rng.normal(size=3)
        np.testing.assert_allclose(O.vee(O.hat(a)), a, atol=0)
        np.testing.assert_allclose(O.hat(a) @ b, np.cross(a, b), atol=1e-15)
        np.testing.assert_allclose(O.hat(a), -O.hat(a).T, atol=0)


def test_quat_to_rot_matches_scipy_and_ignores_scale():
    rng = np.random.default_rng(2)
    for _ in range(20):
        r = Rotation.random(random_state=rng)
        q = quat_wxyz(r)
        np.testing.assert_allclose(O.quat_to_rot(q), r.as_matrix(), atol=1e-14)
        np.testing.assert_allclose(O.quat_to_rot(3.7 * q), r.as_matrix(), atol=1e-14)


# ----------------------------------------------------------- Eqs. 3, 4, 5 --
def test_attitude_error_zero_when_on_target():
    rng = np.random.default_rng(3)
    for _ in range(10):
        Rd = Rotation.random(random_state=rng).as_matrix()
        eR, eW, M = O.attitude_errors(Rd, np.zeros(3), Rd, np.zeros(3), BODY, GAINS)
        np.testing.assert_allclose(eR, 0, atol=1e-15)
        np.testing.assert_allclose(eW, 0, atol=1e-15)
        np.testing.assert_allclose(M, 0, atol=1e-15)


def test_attitude_error_closed_form_sin_theta_n():
    # R = R_d exp(theta n^)  =>  e_R = sin(theta) n   and   R^T R_d = exp(-theta n^)
    rng = np.random.default_rng(4)
    for _ in range(20):
        Rd_rot = Rotation.random(random_state=rng)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        theta = rng.uniform(0.05, 3.0)
        R = (Rd_rot * Rotation.from_rotvec(theta * n)).as_matrix()
        Wd = rng.normal(size=3)
        W = rng.normal(size=3)
        eR, eW, _ = O.attitude_errors(R, W, Rd_rot.as_matrix(), Wd, BODY, GAINS)
        np.testing.assert_allclose(eR, math.sin(theta) * n, atol=1e-13)
        np.testing.assert_allclose(eW, W - Rotation.from_rotvec(-theta * n).apply(Wd), atol=1e-13)


def test_moment_law_closed_form():
    # Omega = 0, Omega_d = 0:  M = -k_R sin(theta) n (gyroscopic term vanishes)
    rng = np.random.default_rng(5)
    kR = GAINS[6:9]
    for _ in range(10):
        Rd = Rotation.random(random_state=rng)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        theta = rng.uniform(0.05, 1.0)
        R = (Rd * Rotation.from_rotvec(theta * n)).as_matrix()
        _, _, M = O.attitude_errors(R, np.zeros(3), Rd.as_matrix(), np.zeros(3), BODY, GAINS)
        np.testing.assert_allclose(M, -kR * math.sin(theta) * n, atol=1e-14)
    # R = R_d, Omega_d = 0: M = -k_Omega Omega + Omega x (J Omega), J diagonal
    W = np.array([0.7, -1.3, 2.1])
    J = BODY[1:]
    _, _, M = O.attitude_errors(np.eye(3), W, np.eye(3), np.zeros(3), BODY, GAINS)
    np.testing.assert_allclose(M, -GAINS[9:12] * W + np.cross(W, J * W), atol=1e-15)


def test_gyroscopic_feedforward_keeps_body_rate_constant():
    # With k_R = k_Omega = 0 the moment law leaves M = Omega x J Omega, which
    # cancels the gyroscopic term of Euler's equation: Omega stays constant in
    # the body frame even for an asymmetric J (drop the term or flip its sign
    # and Omega precesses).
    world = O.World(n_envs=1, motor_tau=0.0, u_max=1e9, kR=(0, 0, 0), kW=(0, 0, 0))
    body = np.array([[0.75], [0.004], [0.007], [0.012]])
    s0 = state13(q=quat_wxyz(Rotation.from_euler("ZYX", [0.3, 0.1, -0.2])), w=(0.4, -0.3, 0.5))
    fl = O.make_fleet(world, state=s0[:, None], body=body, modes=[O.MODE_ATT_THRUST],
                      targets=np.array([[0.0], [0.0], [0.0], [7.0]]))
    fl.motors[:4, 0] = 7.0 / 4
    O.rollout(world, fl, 100)
    np.testing.assert_allclose(fl.state[10:13, 0], s0[10:13], atol=1e-12)


# ----------------------------------------------------------- Eqs. 1 and 2 --
def test_desired_rate_eq2():
    # phi = theta = 0 gives a pure body z rate; in general Omega_d is the body
    # rate of a pure world-z yaw rate seen from R_d = Rz Ry Rx: R_d^T (0,0,psi_dot)
    np.testing.assert_allclose(O.desired_rate(0.0, 0.0, 0.7), [0, 0, 0.7], atol=0)
    rng = np.random.default_rng(6)
    for _ in range(20):
        phi, theta, psi, r = rng.uniform(-1.2, 1.2, size=4)
        Rd = Rotation.from_euler("ZYX", [psi, theta, phi]).as_matrix()
        np.testing.assert_allclose(O.desired_rate(phi, theta, r), Rd.T @ np.array([0, 0, r]), atol=1e-14)


def test_attitude_mode_desired_frame_eq1():
    rng = np.random.default_rng(7)
    for _ in range(20):
        psi, th0, ph0 = rng.uniform(-3.0, 3.0), rng.uniform(-1.2, 1.2), rng.uniform(-1.2, 1.2)
        q = quat_wxyz(Rotation.from_euler("ZYX", [psi, th0, ph0]))
        phi_d, theta_d, rate = rng.uniform(-0.6, 0.6, size=3)
        out = O.controller(O.MODE_ATT_THRUST, state13(q=q), [phi_d, theta_d, rate, 6.0], BODY, GAINS)
        Rd = Rotation.from_euler("ZYX", [psi, theta_d, phi_d]).as_matrix()
        np.testing.assert_allclose(out["Rd"], Rd, atol=1e-13)
        assert out["fM"][0] == 6.0


# ---------------------------------------------------------- Eqs. 6 to 9 --
def test_velocity_mode_tilt_points_thrust_along_commanded_acceleration():
    rng = np.random.default_rng(8)
    for _ in range(30):
        psi = rng.uniform(-3, 3)
        R = Rotation.from_euler("ZYX", [psi, rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5)])
        v = rng.normal(size=3)
        vd = rng.uniform(-2, 2, size=3)
        rate = rng.uniform(-1, 1)
        out = O.controller(O.MODE_BODY_VEL, state13(v=v, q=quat_wxyz(R)), list(vd) + [rate], BODY, GAINS)
        Rpsi = Rotation.from_euler("Z", psi).as_matrix()
        a = GAINS[3:6] * (vd - Rpsi.T @ v) + np.array([0, 0, G])
        # desired thrust axis R_d e3 is the commanded acceleration direction (V frame)
        np.testing.assert_allclose(Rpsi.T @ out["Rd"][:, 2], a / np.linalg.norm(a), atol=1e-13)
        # the desired frame keeps the current yaw: R_d e1 has no V-frame y component
        assert abs((Rpsi.T @ out["Rd"][:, 0])[1]) < 1e-13
        # thrust is m a . b3 (collective thrust projected on the body axis)
        np.testing.assert_allclose(out["fM"][0], BODY[0] * a @ (Rpsi.T @ R.as_matrix()[:, 2]), rtol=1e-13)


def test_velocity_mode_hover_is_equilibrium():
    q = quat_wxyz(Rotation.from_euler("Z", 0.8))
    vd = np.array([0.4, -0.2, 0.1])
    v_world = Rotation.from_euler("Z", 0.8).apply(vd)
    out = O.controller(O.MODE_BODY_VEL, state13(v=v_world, q=q), list(vd) + [0.0], BODY, GAINS)
    np.testing.assert_allclose(out["fM"][0], BODY[0] * G, rtol=1e-14)
    np.testing.assert_allclose(out["fM"][1:], 0, atol=1e-14)


def test_velocity_mode_converges():
    world = O.World(n_envs=1)
    vd = np.array([1.0, -0.5, 0.3])
    s0 = state13(q=quat_wxyz(Rotation.from_euler("Z", 0.5)))
    fl = O.make_fleet(world, state=s0[:, None], modes=[O.MODE_BODY_VEL],
                      targets=np.array([[vd[0]], [vd[1]], [vd[2]], [0.0]]))
    fl.motors[:4, 0] = 0.75 * G / 4
    O.rollout(world, fl, 800)
    q = fl.state[6:10, 0]
    R = O.quat_to_rot(q)
    psi = math.atan2(R[1, 0], R[0, 0])
    vV = Rotation.from_euler("Z", psi).inv().apply(fl.state[3:6, 0])
    np.testing.assert_allclose(vV, vd, atol=1e-3)
    np.testing.assert_allclose(fl.state[10:13, 0], 0, atol=1e-3)


def test_velocity_mode_tracks_yaw_rate():
    world = O.World(n_envs=1)
    fl = O.make_fleet(world, state=state13()[:, None], modes=[O.MODE_BODY_VEL],
                      targets=np.array([[0.0], [0.0], [0.0], [0.5]]))
    fl.motors[:4, 0] = 0.75 * G / 4
    O.rollout(world, fl, 600)
    np.testing.assert_allclose(fl.state[10:13, 0], [0, 0, 0.5], atol=1e-3)


# ---------------------------------------------------------- position mode --
def test_position_mode_hover_equilibrium_and_fixed_point():
    psi_d = 0.7
    pd = np.array([1.0, -2.0, 0.5])
    q = quat_wxyz(Rotation.from_euler("Z", psi_d))
    s0 = state13(p=pd, q=q)
    out = O.controller(O.MODE_POSITION, s0, list(pd) + [psi_d], BODY, GAINS)
    np.testing.assert_allclose(out["fM"][0], BODY[0] * G, rtol=1e-15)
    np.testing.assert_allclose(out["fM"][1:], 0, atol=1e-15)
    W, u = O.allocate(4, out["fM"], np.zeros(4), alpha=1.0)
    np.testing.assert_allclose(u, BODY[0] * G / 4, rtol=1e-14)
    world = O.World(n_envs=1)
    fl = O.make_fleet(world, state=s0[:, None], modes=[O.MODE_POSITION],
                      targets=np.array([[pd[0]], [pd[1]], [pd[2]], [psi_d]]))
    fl.motors[:4, 0] = BODY[0] * G / 4
    O.rollout(world, fl, 100)
    np.testing.assert_allclose(fl.state[:, 0], s0, atol=1e-12)


def test_position_mode_desired_frame_construction():
    rng = np.random.default_rng(9)
    for _ in range(30):
        R = Rotation.random(random_state=rng)
        p, v, pd = rng.normal(size=3), rng.normal(size=3), rng.normal(size=3)
        psi_d = rng.uniform(-3, 3)
        out = O.controller(O.MODE_POSITION, state13(p=p, v=v, q=quat_wxyz(R)), list(pd) + [psi_d], BODY, GAINS)
        Rd = out["Rd"]
        np.testing.assert_allclose(Rd.T @ Rd, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(Rd) - 1) < 1e-14
        a = -GAINS[0:3] * (p - pd) - GAINS[3:6] * v + np.array([0, 0, G])
        np.testing.assert_allclose(Rd[:, 2], a / np.linalg.norm(a), atol=1e-14)
        b1c = np.array([math.cos(psi_d), math.sin(psi_d), 0])
        assert abs(Rd[:, 1] @ b1c) < 1e-14            # b2d is orthogonal to the heading
        assert Rd[:, 0] @ b1c > 0                      # b1d leans towards the heading
        np.testing.assert_allclose(out["Wd"], 0, atol=0)
        np.testing.assert_allclose(out["fM"][0], BODY[0] * a @ R.as_matrix()[:, 2], rtol=1e-13)


def test_position_mode_converges_from_small_errors():
    n = 8
    rng = np.random.default_rng(10)
    world = O.World(n_envs=n)
    st = np.zeros((13, n))
    tg = np.zeros((4, n))
    for i in range(n):
        pd = rng.uniform(-3, 3, size=3)
        psi_d = rng.uniform(-3, 3)
        e = rng.normal(size=3)
        e *= 0.1 / np.linalg.norm(e)
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        R = Rotation.from_euler("Z", psi_d) * Rotation.from_rotvec(math.radians(5) * ax)
        st[:, i] = state13(p=pd + e, q=quat_wxyz(R))
        tg[:, i] = list(pd) + [psi_d]
    fl = O.make_fleet(world, state=st, modes=np.zeros(n), targets=tg)
    fl.motors[:4] = 0.75 * G / 4
    O.rollout(world, fl, 1000)
    ex = fl.state[0:3] - tg[0:3]
    assert np.max(np.linalg.norm(ex, axis=0)) < 1e-3
    for i in range(n):
        R = O.quat_to_rot(fl.state[6:10, i])
        Rd = Rotation.from_euler("Z", tg[3, i]).as_matrix()
        eR = 0.5 * O.vee(Rd.T @ R - R.T @ Rd)
        assert np.linalg.norm(eR) < 1e-3


# ------------------------------------------------------------- allocation --
@pytest.mark.parametrize("n_rot", [4, 6, 8])
def test_allocation_matrix_from_rotor_geometry(n_rot):
    A, Ap = O.rotors(n_rot)
    start = {4: 45.0, 6: 30.0, 8: 22.5}[n_rot]
    for i in range(n_rot):
        beta = math.radians(start + 360.0 * i / n_rot)
        r = 0.13 * np.array([math.cos(beta), math.sin(beta), 0.0])
        spin = 1.0 if i % 2 == 0 else -1.0
        moment = np.cross(r, [0, 0, 1.0]) + spin * 0.016 * np.array([0, 0, 1.0])
        np.testing.assert_allclose(A[:, i], [1.0, moment[0], moment[1], moment[2]], atol=1e-15)
    np.testing.assert_allclose(A @ Ap, np.eye(4), atol=1e-12)
    np.testing.assert_allclose(Ap, np.linalg.pinv(A), atol=1e-12)


@pytest.mark.parametrize("n_rot", [4, 6, 8])
def test_allocation_reproduces_unsaturated_wrench(n_rot):
    cmd = np.array([8.0, 0.05, -0.04, 0.01])
    W, u = O.allocate(n_rot, cmd, np.zeros(n_rot), u_max=5.0, alpha=1.0)
    assert np.all(u > 0) and np.all(u < 5)
    np.testing.assert_allclose(W, cmd, atol=1e-13)


def test_allocation_clamps_each_motor():
    W, u = O.allocate(4, np.array([40.0, 0, 0, 0]), np.zeros(4), u_max=5.0, alpha=1.0)
    np.testing.assert_allclose(u, 5.0, atol=0)
    np.testing.assert_allclose(W[0], 20.0, atol=1e-14)
    W, u = O.allocate(4, np.array([-3.0, 0, 0, 0]), np.ones(4), u_max=5.0, alpha=1.0)
    np.testing.assert_allclose(u, 0.0, atol=0)


def test_motor_lag_step_response():
    tau, h = 0.03, 0.0025
    alpha = 1 - math.exp(-h / tau)
    u = np.zeros(4)
    cmd = np.array([6.0, 0, 0, 0])   # 1.5 N per motor
    for k in range(1, 60):
        _, u = O.allocate(4, cmd, u, u_max=5.0, alpha=alpha)
        np.testing.assert_allclose(u, 1.5 * (1 - math.exp(-k * h / tau)), rtol=1e-12)


# ------------------------------------------------------------- integrators --
def free_fall_world(integrator, drag=0.0, substeps=1):
    return O.World(n_envs=1, integrator=integrator, drag=drag, substeps_per_step=substeps)


def test_free_fall_semi_implicit_euler_discrete_closed_form():
    world = free_fall_world(O.INTEG_SIE)
    p0, v0 = np.array([0.3, -1.0, 2.0]), np.array([1.0, 0.5, 3.0])
    fl = O.make_fleet(world, state=state13(p=p0, v=v0)[:, None], modes=[O.MODE_WRENCH])
    n, d = 37, 0.01
    O.rollout(world, fl, n)
    gv = np.array([0, 0, -G])
    np.testing.assert_allclose(fl.state[3:6, 0], v0 + n * d * gv, atol=1e-12)
    np.testing.assert_allclose(fl.state[0:3, 0], p0 + n * d * v0 + gv * d * d * n * (n + 1) / 2, atol=1e-12)


def test_free_fall_rk4_exact_parabola():
    world = free_fall_world(O.INTEG_RK4, substeps=4)
    p0, v0 = np.array([0.3, -1.0, 2.0]), np.array([1.0, 0.5, 3.0])
    fl = O.make_fleet(world, state=state13(p=p0, v=v0)[:, None], modes=[O.MODE_WRENCH])
    O.rollout(world, fl, 50)
    t = 0.5
    np.testing.assert_allclose(fl.state[0:3, 0], p0 + v0 * t + 0.5 * np.array([0, 0, -G]) * t * t, atol=1e-12)


def test_linear_drag_discrete_closed_form():
    c, m, d = 0.1, 0.75, 0.01
    world = free_fall_world(O.INTEG_SIE, drag=c)
    v0 = np.array([2.0, -1.0, 0.0])
    fl = O.make_fleet(world, state=state13(v=v0)[:, None], modes=[O.MODE_WRENCH])
    n = 200
    O.rollout(world, fl, n)
    v_inf = np.array([0, 0, -G * m / c])
    np.testing.assert_allclose(fl.state[3:6, 0], v_inf + (v0 - v_inf) * (1 - d * c / m) ** n, rtol=1e-11)


def _torque_free(integrator, n_steps, substeps):
    world = O.World(n_envs=1, integrator=integrator, substeps_per_step=substeps)
    body = np.array([[0.75], [0.004], [0.007], [0.012]])
    q0 = quat_wxyz(Rotation.from_euler("ZYX", [0.2, -0.4, 0.9]))
    fl = O.make_fleet(world, state=state13(q=q0, w=(1.5, -2.0, 0.7))[:, None], modes=[O.MODE_WRENCH], body=body)
    O.rollout(world, fl, n_steps)
    return fl, body[1:, 0]


def _momentum_energy(state, J):
    R = O.quat_to_rot(state[6:10])
    W = state[10:13]
    return R @ (J * W), 0.5 * W @ (J * W)


def test_torque_free_rk4_conserves_momentum_energy_and_orthonormality():
    world = O.World(n_envs=1)
    J = np.array([0.004, 0.007, 0.012])
    q0 = quat_wxyz(Rotation.from_euler("ZYX", [0.2, -0.4, 0.9]))
    s0 = state13(q=q0, w=(1.5, -2.0, 0.7))
    L0, E0 = _momentum_energy(s0, J)
    fl, _ = _torque_free(O.INTEG_RK4, 1000, 4)
    L1, E1 = _momentum_energy(fl.state[:, 0], J)
    assert np.linalg.norm(L1 - L0) / np.linalg.norm(L0) < 1e-8
    assert abs(E1 - E0) / E0 < 1e-8
    R = O.quat_to_rot(fl.state[6:10, 0])
    assert np.max(np.abs(R.T @ R - np.eye(3))) < 1e-12
    assert abs(np.linalg.norm(fl.state[6:10, 0]) - 1) < 1e-14
    del world


def test_integrator_orders_of_convergence():
    # Error against a fine RK4 reference at t = 1 s: halving the step divides
    # the RK4 error by ~16 (fourth order) and the Euler error by ~2 (first).
    ref, _ = _torque_free(O.INTEG_RK4, 100, 64)
    def err(integ, sub):
        fl, _ = _torque_free(integ, 100, sub)
        return np.linalg.norm(fl.state[10:13, 0] - ref.state[10:13, 0])
    r_rk4 = err(O.INTEG_RK4, 2) / err(O.INTEG_RK4, 4)
    r_sie = err(O.INTEG_SIE, 8) / err(O.INTEG_SIE, 16)
    assert 12 < r_rk4 < 20, r_rk4
    assert 1.6 < r_sie < 2.4, r_sie


def test_thrust_acts_along_body_z_axis():
    rng = np.random.default_rng(11)
    for integ in (O.INTEG_SIE, O.INTEG_RK4):
        R = Rotation.random(random_state=rng)
        s0 = state13(q=quat_wxyz(R))
        f = 9.0
        out = O.integrate(integ, s0, [f, 0, 0, 0], BODY, 0.0, 1e-3)
        acc = (out[3:6] - s0[3:6]) / 1e-3
        np.testing.assert_allclose(acc, f / BODY[0] * R.apply([0, 0, 1]) + np.array([0, 0, -G]), atol=1e-10)


def test_moment_produces_angular_acceleration_J_inverse():
    s0 = state13()
    M = np.array([0.01, -0.02, 0.003])
    out = O.integrate(O.INTEG_SIE, s0, [0, *M], BODY, 0.0, 1e-3)
    np.testing.assert_allclose((out[10:13] - s0[10:13]) / 1e-3, M / BODY[1:], rtol=1e-12)
    # small rotation about the body axes: q' = 1/2 q (x) (0, Omega)
    s1 = state13(w=(0.2, 0.0, 0.0))
    out = O.integrate(O.INTEG_RK4, s1, [0, 0, 0, 0], BODY, 0.0, 0.5)
    np.testing.assert_allclose(out[6:10], quat_wxyz(Rotation.from_rotvec([0.1, 0, 0])), atol=1e-9)


# --------------------------------------------------------------- collision --
def test_sphere_obb_axis_aligned_faces_edges_corners():
    r = 0.2
    box = np.array([1.0, -2.0, 0.5, 0.5, 0.3, 0.2, 1.0, 0.0, 0.0, 0.0])
    c, h = box[:3], box[3:6]
    eps = 1e-9
    assert O.sphere_obb(c, r, box)                                          # centre inside
    assert O.sphere_obb(c + [h[0] + r - eps, 0, 0], r, box)                   # face
    assert not O.sphere_obb(c + [h[0] + r + eps, 0, 0], r, box)
    assert not O.sphere_obb(c - [0, h[1] + r + eps, 0], r, box)
    d = r / math.sqrt(2)
    assert O.sphere_obb(c + [h[0] + d - eps, 0, h[2] + d - eps], r, box)      # edge
    assert not O.sphere_obb(c + [h[0] + d + eps, 0, h[2] + d + eps], r, box)
    d = r / math.sqrt(3)
    assert O.sphere_obb(c + h + d - eps, r, box)                              # corner
    assert not O.sphere_obb(c + h + d + eps, r, box)


def test_sphere_obb_brute_force_rotated():
    rng = np.random.default_rng(12)
    g = np.linspace(-1, 1, 41)
    unit = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    checked = 0
    for _ in range(60):
        rot = Rotation.random(random_state=rng)
        h = rng.uniform(0.1, 1.0, size=3)
        c = rng.uniform(-1, 1, size=3)
        pts = c + rot.apply(unit * h)               # dense samples filling the box
        spacing = 2 * np.max(h) / 40 * math.sqrt(3)
        box = np.concatenate([c, h, quat_wxyz(rot)])
        for _ in range(20):
            p = c + rng.uniform(-2.0, 2.0, size=3)
            dmin = np.min(np.linalg.norm(pts - p, axis=1))
            if dmin < 0.2 - spacing:
                assert O.sphere_obb(p, 0.2, box)
                checked += 1
            elif dmin > 0.2 + 1e-12 and _outside_margin(p, c, h, rot, 0.2):
                assert not O.sphere_obb(p, 0.2, box)
                checked += 1
    assert checked > 500


def _outside_margin(p, c, h, rot, r):
    # exact distance from the box (independent of the oracle's clamp form):
    # the point in the box frame, distance = norm of the positive excess
    d = rot.inv().apply(p - c)
    excess = np.maximum(np.abs(d) - h, 0.0)
    return np.linalg.norm(excess) > r + 1e-9


# ----------------------------------------------------- Philox and sampler --
def test_philox_known_answer_vectors():
    rows = [ln.split() for ln in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        vals = [int(x, 16) for x in r]
        out = O.philox4x32_10(vals[0:4], vals[4:6])
        assert [int(x) for x in out] == vals[6:10]


def test_own_sincos_and_log_accuracy():
    rng = np.random.default_rng(13)
    for h in np.concatenate([rng.uniform(0, math.pi / 2, 500), [0.0, math.pi / 2 * (1 - 2**-22)]]):
        s, c = O.sincos_poly(np.float32(h))
        hf = float(np.float32(h))
        assert abs(s - math.sin(hf)) < 3e-7 and abs(c - math.cos(hf)) < 3e-7
    for w in rng.integers(0, 2**32, size=500, dtype=np.uint64):
        c, s = O.sincos_turn(int(w))
        ang = 2 * math.pi * (int(w) >> 8) / 2**24
        assert abs(c - math.cos(ang)) < 5e-7 and abs(s - math.sin(ang)) < 5e-7
        lu = O.log_u01(int(w))
        u = ((int(w) >> 8) + 1) / 2**24
        assert abs(lu - math.log(u)) < 2e-6 * max(1.0, abs(math.log(u)))
    assert O.log_u01(0xFFFFFFFF) == 0.0


def test_reset_sampler_distribution():
    from scipy import stats
    n = 20000
    draws = np.stack([O.sample_reset(12345, i, 1 + (i % 3)) for i in range(n)])
    p, v, q = draws[:, 0:3], draws[:, 3:6], draws[:, 6:10].astype(np.float64)
    assert p.min() >= -2.0 and p.max() < 2.0
    for k in range(3):
        assert stats.kstest(p[:, k], stats.uniform(loc=-2, scale=4).cdf).pvalue > 1e-4
        assert stats.kstest(v[:, k], stats.norm(scale=0.5).cdf).pvalue > 1e-4
    np.testing.assert_allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-6)
    angle = 2 * np.arccos(np.clip(q[:, 0], -1, 1))
    assert angle.max() <= math.pi / 6 + 1e-6
    assert stats.kstest(angle, stats.uniform(scale=math.pi / 6).cdf).pvalue > 1e-4
    axis = q[:, 1:] / np.linalg.norm(q[:, 1:], axis=1, keepdims=True)
    for k in range(3):      # uniform on the sphere: each coordinate ~ U[-1, 1]
        assert stats.kstest(axis[:, k], stats.uniform(loc=-1, scale=2).cdf).pvalue > 1e-4
    # different epochs / seeds give different draws
    assert not np.array_equal(O.sample_reset(1, 5, 1), O.sample_reset(1, 5, 2))
    assert not np.array_equal(O.sample_reset(1, 5, 1), O.sample_reset(2, 5, 1))


def test_reset_writes_draw_hover_and_bumps_epoch():
    world = O.World(n_envs=6, n_hexa=2, n_octo=1)
    fl = O.make_fleet(world, seed=77)
    O.reset(world, fl, mask=[1, 0, 1, 1, 0, 1])
    for i in range(6):
        if i in (1, 4):
            assert fl.epoch[i] == 0 and np.all(fl.state[:, i] == 0)
            continue
        assert fl.epoch[i] == 1
        d = O.sample_reset(77, i, 1)
        np.testing.assert_array_equal(fl.state[0:10, i].astype(np.float32), d)
        np.testing.assert_array_equal(fl.state[10:13, i], 0)
        n_rot = [4, 4, 4, 6, 6, 8][i]
        hv = np.float32(np.float32(0.75) * np.float32(9.81)) / np.float32(n_rot)
        np.testing.assert_array_equal(fl.motors[:n_rot, i].astype(np.float32), hv)


def test_collision_resets_with_next_epoch():
    world = O.World(n_envs=2, n_obs=1)
    st = np.zeros((13, 2))
    st[6] = 1.0
    st[0:3, 0] = [0.0, 0.0, 10.0]    # env 0 inside its box, env 1 far away
    st[0:3, 1] = [50.0, 0.0, 0.0]
    boxes = np.zeros((1, 10, 2))
    boxes[0, 0:3, :] = [[0.0, 0.0], [0.0, 0.0], [10.0, 10.0]]
    boxes[0, 3:6, :] = 1.0
    boxes[0, 6, :] = 1.0
    fl = O.make_fleet(world, state=st, modes=[O.MODE_WRENCH] * 2, boxes=boxes, epoch=[4, 4], seed=9)
    collided, resets = O.rollout(world, fl, 1)
    assert list(collided) == [1, 0] and list(resets) == [1, 0]
    assert list(fl.epoch) == [5, 4]
    np.testing.assert_array_equal(fl.state[0:10, 0].astype(np.float32), O.sample_reset(9, 0, 5))


# ----------------------------------------------------- dual numbers / counts --
def test_dual_jvp_matches_central_difference():
    world = O.World(n_envs=1)
    rng = np.random.default_rng(14)
    s0 = state13(p=(0.2, -0.1, 0.3), v=(0.1, 0.2, -0.1), q=quat_wxyz(Rotation.from_euler("ZYX", [0.3, 0.1, -0.1])),
                 w=(0.1, -0.1, 0.05))
    motors = np.full(4, 0.75 * G / 4)
    tgt = [0.5, -0.4, 0.6, 0.2]
    goal = np.array([0.5, -0.4, 0.6])
    ds, dg = rng.normal(size=13), rng.normal(size=12)
    L, dL = O.vehicle_loss_jvp(world, 4, O.MODE_POSITION, tgt, BODY, s0, motors, GAINS, ds, dg, 50, goal)
    eps = 1e-6
    Lp = O.vehicle_loss(world, 4, O.MODE_POSITION, tgt, BODY, s0 + eps * ds, motors, GAINS + eps * dg, 50, goal)
    Lm = O.vehicle_loss(world, 4, O.MODE_POSITION, tgt, BODY, s0 - eps * ds, motors, GAINS - eps * dg, 50, goal)
    assert abs(L - O.vehicle_loss(world, 4, O.MODE_POSITION, tgt, BODY, s0, motors, GAINS, 50, goal)) < 1e-12
    assert abs(dL - (Lp - Lm) / (2 * eps)) < 1e-6 * max(1.0, abs(dL))


@pytest.mark.parametrize("mode,tgt", [
    (O.MODE_POSITION, [0.5, -0.4, 0.6, 0.2]),
    (O.MODE_BODY_VEL, [0.4, -0.3, 0.2, 0.3]),
    (O.MODE_ATT_THRUST, [0.1, -0.15, 0.2, 0.75 * G * 1.05]),
    (O.MODE_WRENCH, [0.75 * G, 0.001, -0.002, 0.0005]),
])
def test_dual_jvp_target_tangent_matches_central_difference(mode, tgt):
    # the tangent seeded on the four targets of every command mode
    world = O.World(n_envs=1)
    rng = np.random.default_rng(15 + mode)
    s0 = state13(p=(0.2, -0.1, 0.3), v=(0.1, 0.2, -0.1), q=quat_wxyz(Rotation.from_euler("ZYX", [0.3, 0.1, -0.1])),
                 w=(0.1, -0.1, 0.05))
    motors = np.full(4, 0.75 * G / 4)
    goal = np.array([0.5, -0.4, 0.6])
    ds, dg, dt = rng.normal(size=13), rng.normal(size=12), rng.normal(size=4)
    L, dL = O.vehicle_loss_jvp(world, 4, mode, tgt, BODY, s0, motors, GAINS, ds, dg, 50, goal, d_tgt4=dt)
    _, dL_no_t = O.vehicle_loss_jvp(world, 4, mode, tgt, BODY, s0, motors, GAINS, ds, dg, 50, goal)
    eps = 1e-6
    t = np.asarray(tgt, dtype=np.float64)
    Lp = O.vehicle_loss(world, 4, mode, t + eps * dt, BODY, s0 + eps * ds, motors, GAINS + eps * dg, 50, goal)
    Lm = O.vehicle_loss(world, 4, mode, t - eps * dt, BODY, s0 - eps * ds, motors, GAINS - eps * dg, 50, goal)
    assert abs(dL - (Lp - Lm) / (2 * eps)) < 1e-6 * max(1.0, abs(dL))
    # the target tangent alone
    Lp = O.vehicle_loss(world, 4, mode, t + eps * dt, BODY, s0, motors, GAINS, 50, goal)
    Lm = O.vehicle_loss(world, 4, mode, t - eps * dt, BODY, s0, motors, GAINS, 50, goal)
    assert abs((dL - dL_no_t) - (Lp - Lm) / (2 * eps)) < 1e-6 * max(1.0, abs(dL))


def test_op_counts_are_plausible():
    sie = O.World(n_envs=1)
    rk4 = O.World(n_envs=1, integrator=O.INTEG_RK4, substeps_per_step=4)
    c_sie = O.count_ops(sie, O.MODE_POSITION, 0)
    c_rk4 = O.count_ops(rk4, O.MODE_POSITION, 0)
    c_obs = O.count_ops(rk4, O.MODE_POSITION, 16)
    tot = lambda c: c["add"] + c["mul"] + c["div"] + c["sqrt"] + c["trans"]
    assert 150 < tot(c_sie) < 1500
    assert tot(c_rk4) > 4 * tot(c_sie)
    per_box = (tot(c_obs) - tot(c_rk4)) / 16
    assert 20 < per_box < 120


def test_op_count_of_one_box_test_matches_a_hand_count():
    # d = R_b^T (p - c), e = d - clamp(d, -h, h), hit iff e.e <= r^2, with R_b
    # formed from the unit quaternion: each diagonal entry 1 - 2 (a a + b b) is
    # 3 mul + 2 add, each off-diagonal 2 (a b -+ c d) is 3 mul + 1 add (27 mul,
    # 12 add); p - c 3 add; R_b^T v 9 mul + 6 add; e 3 add; e.e 3 mul + 2 add;
    # r^2 1 mul. Comparisons (the clamp) are counted apart and left out.
    world = O.World(n_envs=1)
    c0 = O.count_ops(world, O.MODE_WRENCH, 0)
    c1 = O.count_ops(world, O.MODE_WRENCH, 1)
    c5 = O.count_ops(world, O.MODE_WRENCH, 5)
    for c in (c1, c5):
        k = 1 if c is c1 else 5
        assert (c["add"] - c0["add"]) == 26 * k and (c["mul"] - c0["mul"]) == 40 * k
        assert (c["div"], c["sqrt"], c["trans"]) == (c0["div"], c0["sqrt"], c0["trans"])


def test_depth_op_counts_match_a_hand_count():
    # per (pixel, box) pair (ray_slab_depth): d_b = R_b^T d 9 mul + 6 add; per axis
    # t1 = (-h - o) / d and t2 = (h - o) / d, 2 add + 2 div (the sign flip is free):
    # 12 add, 9 mul, 6 div; comparisons: d == 0, two for t1 < t2, t_in < lo, up < t_out
    # per axis (15), then t_in < 0, t_out < t0, t0 < max_range (3).
    # per (camera, box): R_b 27 mul + 12 add, o - c 3 add, R_b^T (o - c) 9 mul + 6 add.
    # per pixel: the two centred pixel coordinates 2 add + 1 div each, R d_c 9 mul + 6 add.
    c = O.count_depth_ops()
    assert c["pair"] == {"add": 12, "mul": 9, "div": 6, "sqrt": 0, "trans": 0, "cmp": 18}
    assert c["box"] == {"add": 21, "mul": 36, "div": 0, "sqrt": 0, "trans": 0, "cmp": 0}
    assert c["ray"] == {"add": 10, "mul": 9, "div": 2, "sqrt": 0, "trans": 0, "cmp": 0}


def test_reverse_op_counter_matches_hand_counts():
    # Every adjoint rule accumulates into each active operand (one add per
    # accumulation). dot(a, b) = a.x b.x + a.y b.y + a.z b.z, all active:
    # forward 3 mul + 2 add; reverse: each product 2 x (1 mul + 1 add), each
    # sum 2 x 1 add -> 6 mul, 10 add.
    fwd, rev = O.count_reverse_primitive(0)
    assert (fwd["mul"], fwd["add"]) == (3, 2)
    assert rev == {"add": 10, "mul": 6, "div": 0, "sqrt": 0, "trans": 0}
    # quat_normalize: n = sqrt(w w + x x + y y + z z), q / n: forward 4 mul +
    # 3 add + 1 sqrt + 4 div. Reverse: 4 squares (both operands the same active
    # value) 8 mul + 8 add; 3 sums 6 add; sqrt 1 mul + 1 div + 1 add; 4 quotients
    # with both operands active 4 x (1 div + 1 mul + 2 add).
    fwd, rev = O.count_reverse_primitive(1)
    assert (fwd["mul"], fwd["add"], fwd["sqrt"], fwd["div"]) == (4, 3, 1, 4)
    assert rev == {"add": 23, "mul": 13, "div": 5, "sqrt": 0, "trans": 0}
    # cross(a, b): 6 products and 3 differences: reverse 12 mul + 12 add + 6 add.
    fwd, rev = O.count_reverse_primitive(2)
    assert (fwd["mul"], fwd["add"]) == (6, 3)
    assert rev == {"add": 18, "mul": 12, "div": 0, "sqrt": 0, "trans": 0}


def test_reverse_count_of_a_step_sees_every_mode_and_airframe():
    # The adjoint of a step is a few times the step itself (the cheap-gradient
    # principle bounds reverse mode by a small constant times the function),
    # it grows with the rotor count, and the trig of the angle modes appears.
    world = O.World(n_envs=1)
    for mode in (O.MODE_POSITION, O.MODE_BODY_VEL, O.MODE_ATT_THRUST, O.MODE_WRENCH):
        tot = {}
        for n_rot in (4, 6, 8):
            fwd, rev = O.count_reverse_ops(world, mode, n_rot)
            f = fwd["add"] + fwd["mul"] + fwd["div"] + fwd["sqrt"] + fwd["trans"]
            r = rev["add"] + rev["mul"] + rev["div"] + rev["sqrt"] + rev["trans"]
            assert 1.5 * f < r < 5 * f
            tot[n_rot] = r
        assert tot[4] < tot[6] < tot[8]
        _, rev = O.count_reverse_ops(world, mode, 4)
        assert (rev["trans"] > 0) == (mode in (O.MODE_POSITION, O.MODE_BODY_VEL, O.MODE_ATT_THRUST))


# ------------------------------------------------- obstacle pose re-draw --
ENV_MIN, ENV_MAX = (-5.0, -4.0, 0.0), (5.0, 4.0, 3.0)


def test_box_pose_locked_dimensions_and_euler_composition():
    rng = np.random.default_rng(20)
    for _ in range(20):
        fixed = list(rng.uniform(-3, 3, 3)) + list(rng.uniform(-3.0, 3.0, 3))
        spec = O.box_rand(lock=0b111111, fixed=fixed)
        out = O.sample_box_pose(7, int(rng.integers(0, 1000)), 1, 0, spec, ENV_MIN, ENV_MAX)
        np.testing.assert_array_equal(out[0:3], np.float32(fixed[0:3]))
        q = quat_wxyz(Rotation.from_euler("ZYX", [fixed[5], fixed[4], fixed[3]]))
        got = out[3:7].astype(np.float64)
        if got @ q < 0:
            got = -got
        np.testing.assert_allclose(got, q, atol=2e-6)


def test_box_pose_bounds_and_uniformity():
    from scipy import stats
    spec = O.box_rand(pos_min=(0.1, 0.0, 0.5), pos_max=(0.9, 0.5, 1.0), euler_min=(-0.3, -0.2, -3.0),
                      euler_max=(0.3, 0.2, 3.0), lock=0b000100, fixed=(0, 0, 1.25, 0, 0, 0))
    draws = np.stack([O.sample_box_pose(3, i, 1 + i % 4, i % 16, spec, ENV_MIN, ENV_MAX) for i in range(5000)])
    lo = np.array(ENV_MIN) + (np.array(ENV_MAX) - np.array(ENV_MIN)) * np.array([0.1, 0.0, 0.5])
    hi = np.array(ENV_MIN) + (np.array(ENV_MAX) - np.array(ENV_MIN)) * np.array([0.9, 0.5, 1.0])
    assert np.all(draws[:, 0:2] >= lo[0:2] - 1e-6) and np.all(draws[:, 0:2] <= hi[0:2] + 1e-6)
    assert np.all(draws[:, 2] == np.float32(1.25))                     # z is locked
    for d in range(2):
        assert stats.kstest(draws[:, d], stats.uniform(loc=lo[d], scale=hi[d] - lo[d]).cdf).pvalue > 1e-4
    q = draws[:, 3:7].astype(np.float64)
    np.testing.assert_allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-6)
    ypr = Rotation.from_quat(np.stack([q[:, 1], q[:, 2], q[:, 3], q[:, 0]], 1)).as_euler("ZYX")
    assert np.all(np.abs(ypr[:, 2]) <= 0.3 + 1e-5) and np.all(np.abs(ypr[:, 1]) <= 0.2 + 1e-5)
    assert stats.kstest(ypr[:, 0], stats.uniform(loc=-3.0, scale=6.0).cdf).pvalue > 1e-4


def test_collision_reset_redraws_the_environments_boxes():
    spec = [O.box_rand(pos_min=(0, 0, 0), pos_max=(1, 1, 1), euler_min=(-1, -1, -1), euler_max=(1, 1, 1))] * 2
    world = O.World(n_envs=2, n_obs=2, env_min=ENV_MIN, env_max=ENV_MAX, box_specs=spec)
    st = np.zeros((13, 2))
    st[6] = 1.0
    st[0:3, 0] = [0.0, 0.0, 1.0]     # env 0 inside its first box, env 1 far from both
    st[0:3, 1] = [50.0, 0.0, 0.0]
    boxes = np.zeros((2, 10, 2))
    boxes[:, 0:3, :] = [[0.0, 0.0], [0.0, 0.0], [1.0, 1.0]]
    boxes[1, 0, :] = 30.0
    boxes[:, 3:6, :] = 0.5
    boxes[:, 6, :] = 1.0
    before = boxes.copy()
    fl = O.make_fleet(world, state=st, modes=[O.MODE_WRENCH] * 2, boxes=boxes, epoch=[2, 2], seed=5)
    collided, _ = O.rollout(world, fl, 1)
    assert list(collided) == [1, 0]
    for k in range(2):
        pose = O.sample_box_pose(5, 0, 3, k, spec[k], ENV_MIN, ENV_MAX)
        np.testing.assert_array_equal(fl.boxes[k, 0:3, 0].astype(np.float32), pose[0:3])
        np.testing.assert_array_equal(fl.boxes[k, 6:10, 0].astype(np.float32), pose[3:7])
        np.testing.assert_array_equal(fl.boxes[k, 3:6, 0], before[k, 3:6, 0])    # extents kept
    np.testing.assert_array_equal(fl.boxes[:, :, 1], before[:, :, 1])            # env 1 untouched


# ------------------------------------------------------------ depth camera --
def _cam_state(p=(0, 0, 0), rot=None):
    q = (1, 0, 0, 0) if rot is None else quat_wxyz(rot)
    return state13(p=p, q=q)[:, None]


def test_depth_axis_aligned_wall_closed_form():
    # a wide box whose near face is the plane x = 3: every pixel sees depth 3
    # (distance along the optical axis), or max_range outside the face
    boxes = np.zeros((1, 10, 1))
    boxes[0, 0:3, 0] = [4.0, 0.0, 0.0]
    boxes[0, 3:6, 0] = [1.0, 50.0, 50.0]
    boxes[0, 6, 0] = 1.0
    img = O.render_depth(_cam_state(), boxes, [0], 16, 12, math.radians(90), 20.0)
    np.testing.assert_allclose(img, 3.0, atol=1e-12)
    # camera offset along body x moves the face closer; yaw by 180 deg looks away
    img = O.render_depth(_cam_state(), boxes, [0], 16, 12, math.radians(90), 20.0, cam_offset=(0.5, 0, 0))
    np.testing.assert_allclose(img, 2.5, atol=1e-12)
    img = O.render_depth(_cam_state(rot=Rotation.from_euler("Z", math.pi)), boxes, [0], 8, 6, 1.0, 20.0)
    np.testing.assert_allclose(img, 20.0)


def test_depth_pixel_geometry_and_inside_box():
    # a thin post at (5, 0, 0): only the central columns see it; the column
    # angle follows the pinhole model with f = (W/2) / tan(hfov/2)
    W, H, hfov = 64, 8, math.radians(60)
    boxes = np.zeros((1, 10, 1))
    boxes[0, 0:3, 0] = [5.0, 0.0, 0.0]
    boxes[0, 3:6, 0] = [0.1, 0.1, 10.0]
    boxes[0, 6, 0] = 1.0
    img = O.render_depth(_cam_state(), boxes, [0], W, H, hfov, 30.0)
    f = 0.5 * W / math.tan(0.5 * hfov)
    for c in range(W):
        y = -(c + 0.5 - 0.5 * W) / f             # ray slope to the left
        hits = abs(y * 4.9) <= 0.1 or abs(y * 5.1) <= 0.1
        assert (img[0, 0, c] < 30.0) == hits
    # a camera inside a box sees depth 0
    boxes[0, 0:3, 0] = [0.0, 0.0, 0.0]
    img = O.render_depth(_cam_state(), boxes, [0], 4, 4, 1.0, 30.0)
    np.testing.assert_array_equal(img, 0.0)


def test_depth_brute_force_ray_march():
    # rotated boxes and a rotated camera: the depth of sampled pixels equals
    # the first point of a fine march along the ray that lies in a box
    rng = np.random.default_rng(21)
    n_obs = 5
    boxes = np.zeros((n_obs, 10, 1))
    for k in range(n_obs):
        boxes[k, 0:3, 0] = rng.uniform([2, -3, -2], [8, 3, 2])
        boxes[k, 3:6, 0] = rng.uniform(0.2, 1.0, 3)
        boxes[k, 6:10, 0] = quat_wxyz(Rotation.random(random_state=rng))
    rot = Rotation.from_euler("ZYX", [0.2, -0.1, 0.15])
    W, H, hfov, rmax = 20, 12, math.radians(80), 12.0
    img = O.render_depth(_cam_state(rot=rot), boxes, [0], W, H, hfov, rmax)
    f = 0.5 * W / math.tan(0.5 * hfov)
    ts = np.linspace(0, rmax, 24001)
    checked = 0
    for r in range(0, H, 3):
        for c in range(0, W, 2):
            d = rot.apply([1.0, -(c + 0.5 - 0.5 * W) / f, -(r + 0.5 - 0.5 * H) / f])
            pts = ts[:, None] * d[None, :]
            inside = np.zeros(len(ts), bool)
            for k in range(n_obs):
                rb = Rotation.from_quat(np.roll(boxes[k, 6:10, 0], -1))
                loc = rb.inv().apply(pts - boxes[k, 0:3, 0])
                inside |= np.all(np.abs(loc) <= boxes[k, 3:6, 0], axis=1)
            t_march = ts[np.argmax(inside)] if inside.any() else rmax
            assert abs(img[0, r, c] - t_march) <= 1.5 * (ts[1] - ts[0]) * np.linalg.norm(d), (r, c)
            checked += 1
    assert checked > 30


# ------------------------------------------------------------ reach task --
def test_reach_task_definition_cases():
    n = 4
    st = np.zeros((13, n))
    st[6] = 1.0
    st[0:3, 0] = [1.0, 2.0, 2.0]          # 3 m from the goal
    st[3:6, 1] = [0.0, 3.0, 4.0]          # at the goal, moving at 5 m/s
    st[6:10, 2] = [-1.0, 0.0, 0.0, 0.0]   # q and -q are the same attitude: obs keeps w >= 0
    st[0, 2] = 3.0                        # collided: the crash penalty alone
    st[0, 3] = 20.0                       # too far away
    goals = np.zeros((3, n))
    obs, rew, done = O.reach_task(st, goals, [0, 0, 1, 0], [0, 0, 0, 0])
    np.testing.assert_allclose(rew, [-3.0, -0.5, -10.0, -20.0])
    assert list(done) == [0, 0, 1, 1]
    np.testing.assert_allclose(obs[6:10, 2], [1.0, 0, 0, 0])
    np.testing.assert_allclose(obs[0:3, 0], [1.0, 2.0, 2.0])
    np.testing.assert_allclose(obs[3:6, 1], [0.0, 3.0, 4.0])
    # the goal is subtracted, not added
    obs2, rew2, _ = O.reach_task(st, goals + np.array([[1.0], [2.0], [2.0]]), [0] * n, [0] * n)
    np.testing.assert_allclose(obs2[0:3, 0], 0.0, atol=1e-15)
    assert rew2[0] == 0.0
    _, _, done = O.reach_task(st, goals, [0] * n, [499, 500, 0, 0])
    assert list(done) == [0, 1, 0, 1]
