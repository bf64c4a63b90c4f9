"""FP64 CPU oracle of the multirotor fleet step — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the cpu_baseline / reference
legs of ``bench.py`` import this package. The product library
(``paper_2305_16510_gb300``) never imports it and shares no code with it.

The arithmetic lives in C++ (``aerial_oracle.hpp``, ``philox_sampler.hpp``,
``scalars.hpp``, ``oracle_capi.cpp``); this module compiles it with g++ and
marshals numpy arrays through ctypes. Every array is structure-of-arrays over
environments (row ``r`` of a ``[rows, n]`` array holds field ``r``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liborc.so")
_SOURCES = ["oracle_capi.cpp", "aerial_oracle.hpp", "philox_sampler.hpp", "scalars.hpp"]
_lock = threading.Lock()
_lib = None

MODE_POSITION, MODE_BODY_VEL, MODE_ATT_THRUST, MODE_WRENCH = 0, 1, 2, 3
INTEG_SIE, INTEG_RK4 = 0, 1


def build(force: bool = False) -> str:
    """Compile liborc.so (g++, -O2, strict FP: -ffp-contract=off)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-pthread", "-o", tmp, os.path.join(_HERE, "oracle_capi.cpp")]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i64p = ctypes.POINTER(ctypes.c_longlong)


def _declare(L: ctypes.CDLL) -> None:
    vp = ctypes.c_void_p
    L.orc_world_size.restype = ctypes.c_int
    L.orc_rollout.argtypes = [vp, ctypes.c_int, _dp, _dp, _dp, _u8p, _dp, _dp, _u32p, ctypes.c_uint64, _u8p,
                              _u32p, _u32p, ctypes.c_int]
    L.orc_reset.argtypes = [vp, _u8p, ctypes.c_uint64, _dp, _dp, _dp, _u32p, _u32p, _dp]
    L.orc_box_rand_size.restype = ctypes.c_int
    L.orc_reach_task.argtypes = [ctypes.c_int, _dp, _dp, _u8p, _u32p, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_uint32, _dp, _dp, _u8p]
    L.orc_render_depth.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_int, _u32p, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp]
    L.orc_sample_box_pose.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, vp, _fp,
                                      _fp, _fp]
    L.orc_hat.argtypes = [_dp, _dp]
    L.orc_vee.argtypes = [_dp, _dp]
    L.orc_quat_to_rot.argtypes = [_dp, _dp]
    L.orc_attitude_errors.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_desired_rate.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp]
    L.orc_controller.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_rotors.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp]
    L.orc_allocate.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp, ctypes.c_double,
                               ctypes.c_double, _dp]
    L.orc_integrate.argtypes = [ctypes.c_int, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp]
    L.orc_sphere_obb.argtypes = [_dp, ctypes.c_double, _dp]
    L.orc_sphere_obb.restype = ctypes.c_int
    L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
    L.orc_sample_reset.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _fp]
    L.orc_hover_thrust.argtypes = [ctypes.c_float, ctypes.c_int]
    L.orc_hover_thrust.restype = ctypes.c_float
    L.orc_sincos_poly.argtypes = [ctypes.c_float, _fp, _fp]
    L.orc_sincos_turn.argtypes = [ctypes.c_uint32, _fp, _fp]
    L.orc_log_u01.argtypes = [ctypes.c_uint32]
    L.orc_log_u01.restype = ctypes.c_float
    L.orc_count_ops.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i64p]
    L.orc_count_depth_ops.argtypes = [_i64p, _i64p, _i64p]
    L.orc_count_reverse_ops.argtypes = [vp, ctypes.c_int, ctypes.c_int, _i64p, _i64p]
    L.orc_count_reverse_primitive.argtypes = [ctypes.c_int, _i64p, _i64p]
    L.orc_vehicle_loss.argtypes = [vp, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, ctypes.c_int, _dp,
                                   ctypes.c_double, ctypes.c_double]
    L.orc_vehicle_loss.restype = ctypes.c_double
    L.orc_vehicle_loss_jvp.argtypes = [vp, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                       ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double, _dp]
    L.orc_vehicle_loss_jvp.restype = ctypes.c_double


class _World(ctypes.Structure):
    _fields_ = [("n_envs", ctypes.c_int32), ("substeps_per_step", ctypes.c_int32),
                ("integrator", ctypes.c_int32), ("n_obs", ctypes.c_int32),
                ("n_quad", ctypes.c_int32), ("n_hexa", ctypes.c_int32), ("n_octo", ctypes.c_int32),
                ("pad_", ctypes.c_int32),
                ("dt", ctypes.c_double), ("motor_tau", ctypes.c_double), ("drag", ctypes.c_double),
                ("sphere_r", ctypes.c_double), ("u_max", ctypes.c_double), ("arm", ctypes.c_double),
                ("k_yaw", ctypes.c_double),
                ("kx", ctypes.c_double * 3), ("kv", ctypes.c_double * 3), ("kR", ctypes.c_double * 3),
                ("kW", ctypes.c_double * 3), ("box_rand", ctypes.c_void_p)]


class BoxRand(ctypes.Structure):
    """Re-draw spec of one obstacle (mirrors the oracle's C struct)."""
    _fields_ = [("pos_min", ctypes.c_float * 3), ("pos_max", ctypes.c_float * 3),
                ("euler_min", ctypes.c_float * 3), ("euler_max", ctypes.c_float * 3),
                ("lock", ctypes.c_uint32), ("fixed", ctypes.c_float * 6)]


class _BoxRandSpec(ctypes.Structure):
    _fields_ = [("env_min", ctypes.c_float * 3), ("env_max", ctypes.c_float * 3), ("per_box", ctypes.c_void_p)]


def box_rand(pos_min=(0, 0, 0), pos_max=(1, 1, 1), euler_min=(0, 0, 0), euler_max=(0, 0, 0), lock=0,
             fixed=(0, 0, 0, 0, 0, 0)) -> BoxRand:
    r = BoxRand()
    r.pos_min[:], r.pos_max[:] = list(pos_min), list(pos_max)
    r.euler_min[:], r.euler_max[:] = list(euler_min), list(euler_max)
    r.lock = lock
    r.fixed[:] = list(fixed)
    return r


@dataclass
class World:
    """Fleet-wide constants of a rollout (mirrors the oracle's C struct)."""
    n_envs: int
    substeps_per_step: int = 1
    integrator: int = INTEG_SIE
    n_obs: int = 0
    n_quad: int | None = None
    n_hexa: int = 0
    n_octo: int = 0
    dt: float = 0.01
    motor_tau: float = 0.03
    drag: float = 0.0
    sphere_r: float = 0.2
    u_max: float = 5.0
    arm: float = 0.13
    k_yaw: float = 0.016
    kx: tuple = (2.0, 2.0, 3.0)
    kv: tuple = (2.0, 2.0, 2.0)
    kR: tuple = (1.2, 1.2, 0.6)
    kW: tuple = (0.2, 0.2, 0.1)
    env_min: tuple | None = None       # obstacle re-draw on reset: environment bounds
    env_max: tuple | None = None
    box_specs: list | None = None      # one BoxRand per obstacle (None: obstacles keep their poses)

    def c(self) -> _World:
        n_quad = self.n_envs - self.n_hexa - self.n_octo if self.n_quad is None else self.n_quad
        w = _World(self.n_envs, self.substeps_per_step, self.integrator, self.n_obs, n_quad, self.n_hexa,
                   self.n_octo, 0, self.dt, self.motor_tau, self.drag, self.sphere_r, self.u_max, self.arm,
                   self.k_yaw)
        w.kx[:] = list(self.kx)
        w.kv[:] = list(self.kv)
        w.kR[:] = list(self.kR)
        w.kW[:] = list(self.kW)
        if self.box_specs:
            arr = (BoxRand * len(self.box_specs))(*self.box_specs)
            spec = _BoxRandSpec()
            spec.env_min[:], spec.env_max[:] = list(self.env_min), list(self.env_max)
            spec.per_box = ctypes.addressof(arr)
            w.box_rand = ctypes.addressof(spec)
            w._keep = (arr, spec)       # keep the structures alive with the World
        assert ctypes.sizeof(w) == lib().orc_world_size()
        return w

    def gains12(self) -> np.ndarray:
        return np.array(list(self.kx) + list(self.kv) + list(self.kR) + list(self.kW), dtype=np.float64)

    def rotor_counts(self) -> np.ndarray:
        n_quad = self.n_envs - self.n_hexa - self.n_octo if self.n_quad is None else self.n_quad
        out = np.full(self.n_envs, 8, dtype=np.int32)
        out[:n_quad] = 4
        out[n_quad:n_quad + self.n_hexa] = 6
        return out


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ct) if a is not None else None


def _f64(a, shape=None) -> np.ndarray:
    out = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        out = out.reshape(shape)
    return out


@dataclass
class Fleet:
    """Mutable FP64 fleet state of the oracle (all arrays SoA)."""
    state: np.ndarray             # [13, n]
    motors: np.ndarray            # [8, n]
    body: np.ndarray              # [4, n]
    modes: np.ndarray             # [n] uint8
    targets: np.ndarray           # [4, n]
    epoch: np.ndarray             # [n] uint32
    boxes: np.ndarray | None = None  # [n_obs, 10, n]
    seed: int = 0
    extra: dict = field(default_factory=dict)


def make_fleet(world: World, *, state=None, motors=None, body=None, modes=None, targets=None, epoch=None,
               boxes=None, seed=0) -> Fleet:
    n = world.n_envs
    body = _f64(body if body is not None else np.tile(np.array([[0.75], [0.007], [0.007], [0.012]]), (1, n)),
                (4, n))
    fl = Fleet(state=_f64(state if state is not None else np.zeros((13, n)), (13, n)).copy(),
               motors=_f64(motors if motors is not None else np.zeros((8, n)), (8, n)).copy(),
               body=body,
               modes=np.ascontiguousarray(np.asarray(modes if modes is not None else np.zeros(n), dtype=np.uint8)),
               targets=_f64(targets if targets is not None else np.zeros((4, n)), (4, n)),
               epoch=np.ascontiguousarray(np.asarray(epoch if epoch is not None else np.zeros(n), dtype=np.uint32)).copy(),
               boxes=None if boxes is None else _f64(boxes, (world.n_obs, 10, n)),
               seed=seed)
    return fl


def rollout(world: World, fleet: Fleet, n_steps: int, n_threads: int = 1, env_ids=None):
    """Advances the fleet in place; returns (collided uint8[n], n_resets uint32[n]).

    env_ids: Philox environment number of each row (default: the row index).
    """
    L = lib()
    ids = None if env_ids is None else np.ascontiguousarray(np.asarray(env_ids, dtype=np.uint32))
    n = world.n_envs
    collided = np.zeros(n, dtype=np.uint8)
    resets = np.zeros(n, dtype=np.uint32)
    boxes = fleet.boxes if fleet.boxes is not None else np.zeros(1)
    w = world.c()
    rc = L.orc_rollout(ctypes.byref(w), int(n_steps), _ptr(fleet.state, _dp), _ptr(fleet.motors, _dp),
                       _ptr(fleet.body, _dp), _ptr(fleet.modes, _u8p), _ptr(fleet.targets, _dp), _ptr(boxes, _dp),
                       _ptr(fleet.epoch, _u32p), ctypes.c_uint64(fleet.seed), _ptr(collided, _u8p),
                       _ptr(resets, _u32p), _ptr(ids, _u32p), int(n_threads))
    if rc != 0:
        raise ValueError(f"orc_rollout failed ({rc})")
    return collided, resets


def reset(world: World, fleet: Fleet, mask=None, seed: int | None = None, env_ids=None) -> None:
    """Resets masked environments in place (all when mask is None).

    env_ids: Philox environment number of each row (default: the row index).
    """
    L = lib()
    if seed is not None:
        fleet.seed = int(seed)
    m = None if mask is None else np.ascontiguousarray(np.asarray(mask, dtype=np.uint8))
    ids = None if env_ids is None else np.ascontiguousarray(np.asarray(env_ids, dtype=np.uint32))
    w = world.c()
    L.orc_reset(ctypes.byref(w), _ptr(m, _u8p), ctypes.c_uint64(fleet.seed), _ptr(fleet.body, _dp),
                _ptr(fleet.state, _dp), _ptr(fleet.motors, _dp), _ptr(fleet.epoch, _u32p), _ptr(ids, _u32p),
                _ptr(fleet.boxes, _dp))


# ------------------------------------------------------------ single pieces --
def hat(a):
    out = np.zeros(9)
    lib().orc_hat(_ptr(_f64(a), _dp), _ptr(out, _dp))
    return out.reshape(3, 3)


def vee(m):
    out = np.zeros(3)
    lib().orc_vee(_ptr(_f64(m, (9,)), _dp), _ptr(out, _dp))
    return out


def quat_to_rot(q):
    out = np.zeros(9)
    lib().orc_quat_to_rot(_ptr(_f64(q), _dp), _ptr(out, _dp))
    return out.reshape(3, 3)


def attitude_errors(R, W, Rd, Wd, body4, gains12):
    eR, eW, M = np.zeros(3), np.zeros(3), np.zeros(3)
    lib().orc_attitude_errors(_ptr(_f64(R, (9,)), _dp), _ptr(_f64(W), _dp), _ptr(_f64(Rd, (9,)), _dp),
                              _ptr(_f64(Wd), _dp), _ptr(_f64(body4), _dp), _ptr(_f64(gains12), _dp),
                              _ptr(eR, _dp), _ptr(eW, _dp), _ptr(M, _dp))
    return eR, eW, M


def desired_rate(phi, theta, yaw_rate):
    out = np.zeros(3)
    lib().orc_desired_rate(float(phi), float(theta), float(yaw_rate), _ptr(out, _dp))
    return out


def controller(mode, state13, tgt4, body4, gains12):
    """Returns dict(fM, Rd, Wd, eR, eW) of one controller evaluation."""
    fM, Rd, Wd, eR, eW = np.zeros(4), np.zeros(9), np.zeros(3), np.zeros(3), np.zeros(3)
    lib().orc_controller(int(mode), _ptr(_f64(state13), _dp), _ptr(_f64(tgt4), _dp), _ptr(_f64(body4), _dp),
                         _ptr(_f64(gains12), _dp), _ptr(fM, _dp), _ptr(Rd, _dp), _ptr(Wd, _dp), _ptr(eR, _dp),
                         _ptr(eW, _dp))
    return {"fM": fM, "Rd": Rd.reshape(3, 3), "Wd": Wd, "eR": eR, "eW": eW}


def rotors(n_rot, arm=0.13, k_yaw=0.016):
    A, Ap = np.zeros(32), np.zeros(32)
    lib().orc_rotors(int(n_rot), float(arm), float(k_yaw), _ptr(A, _dp), _ptr(Ap, _dp))
    return A.reshape(4, 8)[:, :n_rot].copy(), Ap.reshape(8, 4)[:n_rot].copy()


def allocate(n_rot, cmd4, u, u_max=5.0, alpha=1.0, arm=0.13, k_yaw=0.016):
    uu = np.zeros(8)
    uu[:n_rot] = u
    W = np.zeros(4)
    lib().orc_allocate(int(n_rot), float(arm), float(k_yaw), _ptr(_f64(cmd4), _dp), _ptr(uu, _dp),
                       float(u_max), float(alpha), _ptr(W, _dp))
    return W, uu[:n_rot].copy()


def integrate(integrator, state13, W4, body4, drag, h):
    out = np.zeros(13)
    lib().orc_integrate(int(integrator), _ptr(_f64(state13), _dp), _ptr(_f64(W4), _dp), _ptr(_f64(body4), _dp),
                        float(drag), float(h), _ptr(out, _dp))
    return out


def sphere_obb(p, r, box10) -> bool:
    return bool(lib().orc_sphere_obb(_ptr(_f64(p), _dp), float(r), _ptr(_f64(box10), _dp)))


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, _u32p), _ptr(k, _u32p), _ptr(out, _u32p))
    return out


def sample_reset(seed, env, epoch) -> np.ndarray:
    """float32[10]: p xyz, v xyz, q wxyz of the reset draw."""
    out = np.zeros(10, dtype=np.float32)
    lib().orc_sample_reset(ctypes.c_uint64(seed), int(env), int(epoch), _ptr(out, _fp))
    return out


def sample_box_pose(seed, env, epoch, k, spec: BoxRand, env_min, env_max) -> np.ndarray:
    """float32[7]: centre xyz, q wxyz of one obstacle re-draw."""
    lo = np.ascontiguousarray(np.asarray(env_min, dtype=np.float32))
    hi = np.ascontiguousarray(np.asarray(env_max, dtype=np.float32))
    out = np.zeros(7, dtype=np.float32)
    lib().orc_sample_box_pose(ctypes.c_uint64(seed), int(env), int(epoch), int(k), ctypes.byref(spec),
                              _ptr(lo, _fp), _ptr(hi, _fp), _ptr(out, _fp))
    return out


def render_depth(state, boxes, env_ids, width, height, hfov, max_range, cam_offset=(0.0, 0.0, 0.0)):
    """float64 [n_cams, H, W] depth images (see ray_box_depth for the camera model)."""
    st = _f64(state)
    n = st.shape[1]
    bx = _f64(boxes) if boxes is not None and np.asarray(boxes).size else np.zeros(1)
    n_obs = 0 if boxes is None else np.asarray(boxes).shape[0]
    ids = np.ascontiguousarray(np.asarray(env_ids, dtype=np.uint32))
    out = np.zeros((len(ids), height, width))
    lib().orc_render_depth(int(n), int(n_obs), _ptr(st, _dp), _ptr(bx, _dp), len(ids), _ptr(ids, _u32p), int(width),
                           int(height), float(hfov), float(max_range), _ptr(_f64(cam_offset), _dp), _ptr(out, _dp))
    return out


def reach_task(state, goals, collided, steps, w_v=0.1, w_w=0.01, crash=10.0, max_dist=8.0, max_steps=500):
    """(obs [13, n], reward [n], done [n]) of the reach-a-setpoint task."""
    st, g = _f64(state), _f64(goals)
    n = st.shape[1]
    col = np.ascontiguousarray(np.asarray(collided, dtype=np.uint8))
    stp = np.ascontiguousarray(np.asarray(steps, dtype=np.uint32))
    obs, rew, done = np.zeros((13, n)), np.zeros(n), np.zeros(n, np.uint8)
    lib().orc_reach_task(int(n), _ptr(st, _dp), _ptr(g, _dp), _ptr(col, _u8p), _ptr(stp, _u32p), float(w_v),
                         float(w_w), float(crash), float(max_dist), int(max_steps), _ptr(obs, _dp), _ptr(rew, _dp),
                         _ptr(done, _u8p))
    return obs, rew, done


def hover_thrust(m, n_rot) -> np.float32:
    return np.float32(lib().orc_hover_thrust(ctypes.c_float(m), int(n_rot)))


def sincos_poly(h):
    s, c = ctypes.c_float(), ctypes.c_float()
    lib().orc_sincos_poly(ctypes.c_float(h), ctypes.byref(s), ctypes.byref(c))
    return np.float32(s.value), np.float32(c.value)


def sincos_turn(w):
    c, s = ctypes.c_float(), ctypes.c_float()
    lib().orc_sincos_turn(int(w), ctypes.byref(c), ctypes.byref(s))
    return np.float32(c.value), np.float32(s.value)


def log_u01(w) -> np.float32:
    return np.float32(lib().orc_log_u01(int(w)))


def count_ops(world: World, mode: int, n_obs: int, n_rot: int = 4) -> dict:
    """Operations of one step of one vehicle (substeps_per_step substeps, then n_obs box tests)."""
    out = np.zeros(6, dtype=np.int64)
    w = world.c()
    lib().orc_count_ops(ctypes.byref(w), int(mode), int(n_obs), int(n_rot), _ptr(out, _i64p))
    return dict(zip(["add", "mul", "div", "sqrt", "trans", "cmp"], (int(x) for x in out)))


_FWD_KEYS = ["add", "mul", "div", "sqrt", "trans", "cmp"]
_REV_KEYS = ["add", "mul", "div", "sqrt", "trans"]


def count_depth_ops() -> dict:
    """Operations of the depth caster by what they repeat over: 'ray' per
    pixel, 'box' per (camera, box) pair, 'pair' per (pixel, box) pair."""
    outs = [np.zeros(6, dtype=np.int64) for _ in range(3)]
    lib().orc_count_depth_ops(*(_ptr(o, _i64p) for o in outs))
    return {k: dict(zip(_FWD_KEYS, (int(x) for x in o))) for k, o in zip(("ray", "box", "pair"), outs)}


def count_reverse_ops(world: World, mode: int, n_rot: int = 4) -> tuple[dict, dict]:
    """(forward, reverse) operations of one step of the rollout objective with
    state, motors, gains and targets active (see CntRev in scalars.hpp)."""
    fwd, rev = np.zeros(6, dtype=np.int64), np.zeros(5, dtype=np.int64)
    w = world.c()
    lib().orc_count_reverse_ops(ctypes.byref(w), int(mode), int(n_rot), _ptr(fwd, _i64p), _ptr(rev, _i64p))
    return dict(zip(_FWD_KEYS, (int(x) for x in fwd))), dict(zip(_REV_KEYS, (int(x) for x in rev)))


def count_reverse_primitive(which: int) -> tuple[dict, dict]:
    """(forward, reverse) operations of 0 dot(a, b), 1 quat_normalize(q) or
    2 cross(a, b) with every input active."""
    fwd, rev = np.zeros(6, dtype=np.int64), np.zeros(5, dtype=np.int64)
    lib().orc_count_reverse_primitive(int(which), _ptr(fwd, _i64p), _ptr(rev, _i64p))
    return dict(zip(_FWD_KEYS, (int(x) for x in fwd))), dict(zip(_REV_KEYS, (int(x) for x in rev)))


def vehicle_loss(world: World, n_rot, mode, tgt4, body4, state13, motors, gains12, horizon, p_goal,
                 w_pos=1.0, w_omega=0.01) -> float:
    mot = np.zeros(8)
    mot[:len(motors)] = motors
    w = world.c()
    return float(lib().orc_vehicle_loss(ctypes.byref(w), int(n_rot), int(mode), _ptr(_f64(tgt4), _dp),
                                        _ptr(_f64(body4), _dp), _ptr(_f64(state13), _dp), _ptr(mot, _dp),
                                        _ptr(_f64(gains12), _dp), int(horizon), _ptr(_f64(p_goal), _dp),
                                        float(w_pos), float(w_omega)))


def vehicle_loss_jvp(world: World, n_rot, mode, tgt4, body4, state13, motors, gains12, d_state13, d_gains12,
                     horizon, p_goal, w_pos=1.0, w_omega=0.01, d_tgt4=None):
    """(loss, directional derivative along (d_state13, d_gains12, d_tgt4)); d_tgt4 None holds the targets."""
    dt = None if d_tgt4 is None else _f64(d_tgt4)
    mot = np.zeros(8)
    mot[:len(motors)] = motors
    dl = ctypes.c_double()
    w = world.c()
    L = lib().orc_vehicle_loss_jvp(ctypes.byref(w), int(n_rot), int(mode), _ptr(_f64(tgt4), _dp),
                                   _ptr(_f64(body4), _dp), _ptr(_f64(state13), _dp), _ptr(mot, _dp),
                                   _ptr(_f64(gains12), _dp), _ptr(_f64(d_state13), _dp), _ptr(_f64(d_gains12), _dp),
                                   _ptr(dt, _dp), int(horizon), _ptr(_f64(p_goal), _dp), float(w_pos), float(w_omega),
                                   ctypes.byref(dl))
    return float(L), float(dl.value)
