"""ctypes binding of include/ag.h — argument marshalling only.

Every function here has the name of the C entry point it calls and does no
simulation work: it converts Python arguments (ints, torch tensors, numpy
arrays, None) to pointers, calls libaerialgb, and turns a non-zero ag_status
into an AgError carrying ag_last_error(). The library must have been built
(``paper_2305_16510_gb300.build.build()``); if it is missing this module
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

AG_OK, AG_ERR_INVALID, AG_ERR_OOM, AG_ERR_CUDA, AG_ERR_STATE, AG_ERR_TIMEOUT, AG_ERR_UNSUPPORTED = range(7)
AG_MODE_POSITION, AG_MODE_BODY_VEL, AG_MODE_ATT_THRUST, AG_MODE_WRENCH = range(4)
AG_INTEG_SIE, AG_INTEG_RK4 = 0, 1
AG_MAX_OBSTACLES = 64
AG_MAX_ENVS = 1 << 28
STATUS_NAMES = {0: "AG_OK", 1: "AG_ERR_INVALID", 2: "AG_ERR_OOM", 3: "AG_ERR_CUDA", 4: "AG_ERR_STATE",
                5: "AG_ERR_TIMEOUT", 6: "AG_ERR_UNSUPPORTED"}


class AgError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where} -> {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class ag_config(ctypes.Structure):
    _fields_ = [("n_envs", ctypes.c_uint32), ("substeps_per_step", ctypes.c_uint32),
                ("integrator", ctypes.c_uint32), ("n_obstacles", ctypes.c_uint32),
                ("n_quad", ctypes.c_uint32), ("n_hexa", ctypes.c_uint32), ("n_octo", ctypes.c_uint32),
                ("record_every", ctypes.c_uint32),
                ("dt", ctypes.c_float), ("motor_tau", ctypes.c_float), ("drag", ctypes.c_float),
                ("sphere_r", ctypes.c_float), ("u_max", ctypes.c_float), ("arm", ctypes.c_float),
                ("k_yaw", ctypes.c_float), ("mass", ctypes.c_float), ("inertia", ctypes.c_float * 3),
                ("kx", ctypes.c_float * 3), ("kv", ctypes.c_float * 3), ("kR", ctypes.c_float * 3),
                ("kW", ctypes.c_float * 3), ("seed", ctypes.c_uint64), ("hbm_budget_bytes", ctypes.c_uint64)]


class ag_box_randomization(ctypes.Structure):
    _fields_ = [("pos_min", ctypes.c_float * 3), ("pos_max", ctypes.c_float * 3),
                ("euler_min", ctypes.c_float * 3), ("euler_max", ctypes.c_float * 3),
                ("lock", ctypes.c_uint32), ("fixed", ctypes.c_float * 6)]


class ag_reach_config(ctypes.Structure):
    _fields_ = [("command_mode", ctypes.c_uint32), ("action_scale", ctypes.c_float * 4),
                ("action_offset", ctypes.c_float * 4), ("w_v", ctypes.c_float), ("w_omega", ctypes.c_float),
                ("crash", ctypes.c_float), ("max_dist", ctypes.c_float), ("max_steps", ctypes.c_uint32)]


class ag_server_config(ctypes.Structure):
    _fields_ = [("physics", ag_config), ("max_active", ctypes.c_uint32), ("chunk_steps", ctypes.c_uint32),
                ("hbm_budget_bytes", ctypes.c_uint64)]


class ag_request(ctypes.Structure):
    _fields_ = [("n_envs", ctypes.c_uint32), ("n_steps", ctypes.c_uint32), ("n_obstacles", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("seed", ctypes.c_uint64), ("modes", ctypes.c_void_p),
                ("targets", ctypes.c_void_p), ("body", ctypes.c_void_p), ("boxes", ctypes.c_void_p),
                ("pitch", ctypes.c_uint64)]


class ag_server_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("pending", ctypes.c_uint64),
                ("active", ctypes.c_uint64), ("vehicle_steps", ctypes.c_double), ("gpu_ms", ctypes.c_double),
                ("hbm_used_bytes", ctypes.c_uint64)]


class ag_fp32_peak(ctypes.Structure):
    _fields_ = [("scalar_tflops", ctypes.c_double), ("packed_tflops", ctypes.c_double),
                ("scalar_ms", ctypes.c_double), ("packed_ms", ctypes.c_double), ("grid", ctypes.c_uint32),
                ("block", ctypes.c_uint32)]


class ag_alu_peak(ctypes.Structure):
    _fields_ = [("sm_count", ctypes.c_uint32), ("fp32_lanes_per_sm", ctypes.c_uint32),
                ("max_sm_clock_khz", ctypes.c_uint32), ("cc_major", ctypes.c_uint32), ("cc_minor", ctypes.c_uint32),
                ("tflops", ctypes.c_double)]


_lock = threading.Lock()
_lib = None

# every symbol include/*.h declares, with (restype, argtypes)
_vp = ctypes.c_void_p
SIGNATURES = {
    "ag_abi_version": (ctypes.c_int, []),
    "ag_config_default": (None, [ctypes.POINTER(ag_config)]),
    "ag_create": (ctypes.c_int, [ctypes.POINTER(ag_config), _vp, ctypes.POINTER(_vp)]),
    "ag_destroy": (ctypes.c_int, [_vp]),
    "ag_set_commands": (ctypes.c_int, [_vp, _vp, _vp]),
    "ag_set_obstacles": (ctypes.c_int, [_vp, _vp]),
    "ag_set_body": (ctypes.c_int, [_vp, _vp]),
    "ag_get_obstacles": (ctypes.c_int, [_vp, _vp]),
    "ag_render_depth": (ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_float, ctypes.c_float,
                                       ctypes.POINTER(ctypes.c_float * 3), _vp, ctypes.c_uint32, _vp]),
    "ag_set_obstacle_randomization": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_float * 3),
                                                     ctypes.POINTER(ctypes.c_float * 3), _vp]),
    "ag_step": (ctypes.c_int, [_vp, ctypes.c_uint32]),
    "ag_step_plain": (ctypes.c_int, [_vp, ctypes.c_uint32]),
    "ag_reset": (ctypes.c_int, [_vp, _vp, ctypes.c_uint64]),
    "ag_eval_controller": (ctypes.c_int, [_vp, _vp, _vp]),
    "ag_inject_failure": (ctypes.c_int, [_vp, ctypes.c_char_p]),
    "ag_measure_fp32_peak": (ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ag_fp32_peak)]),
    "ag_query_alu_peak": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ag_alu_peak)]),
    "ag_collision_tests_run": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint64)]),
    "ag_render_depth_ieee": (ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_float, ctypes.c_float,
                                            ctypes.POINTER(ctypes.c_float * 3), _vp, ctypes.c_uint32, _vp]),
    "ag_depth_live_pairs": (ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_float, ctypes.c_float,
                                           ctypes.POINTER(ctypes.c_float * 3), _vp, ctypes.c_uint32,
                                           ctypes.POINTER(ctypes.c_uint64)]),
    "ag_get_state": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_uint32)]),
    "ag_get_motors": (ctypes.c_int, [_vp, _vp, _vp]),
    "ag_set_state": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "ag_synchronize": (ctypes.c_int, [_vp]),
    "ag_get_config": (ctypes.c_int, [_vp, ctypes.POINTER(ag_config)]),
    "ag_last_error": (ctypes.c_char_p, [_vp]),
    "ag_set_gains": (ctypes.c_int, [_vp, _vp]),
    "ag_rollout_loss": (ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.c_float, ctypes.c_float, _vp, _vp, _vp]),
    "ag_backward": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "ag_reach_config_default": (None, [ctypes.POINTER(ag_reach_config)]),
    "ag_reach_begin": (ctypes.c_int, [_vp, ctypes.POINTER(ag_reach_config), _vp]),
    "ag_reach_step": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "ag_reach_observe": (ctypes.c_int, [_vp, _vp]),
    "ag_server_config_default": (None, [ctypes.POINTER(ag_server_config)]),
    "ag_server_create": (ctypes.c_int, [ctypes.POINTER(ag_server_config), ctypes.POINTER(_vp)]),
    "ag_server_submit": (ctypes.c_int, [_vp, ctypes.POINTER(ag_request), ctypes.POINTER(ctypes.c_uint64)]),
    "ag_server_wait": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_double, _vp, _vp,
                                      ctypes.POINTER(ctypes.c_double)]),
    "ag_server_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(ag_server_stats)]),
    "ag_server_destroy": (ctypes.c_int, [_vp]),
    "ag_step_plain_noalloc": (ctypes.c_int, [ctypes.POINTER(ag_config), _vp, ctypes.c_uint32, ctypes.c_uint64,
                                             _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_char_p,
                                             ctypes.c_size_t]),
}


ABI_VERSION = 2  # AG_ABI_VERSION of include/ag.h these signatures describe


def library_path() -> str:
    return _build.LIB_PATH


def lib() -> ctypes.CDLL:
    """Loads libaerialgb.so (built in-tree). Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB_PATH
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: run paper_2305_16510_gb300.build.build() "
                                   "(there is no CPU fallback)")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            if L.ag_abi_version() != ABI_VERSION:
                raise RuntimeError(f"{path} implements ABI {L.ag_abi_version()}, this binding ABI {ABI_VERSION}: "
                                   "rebuild it")
            _lib = L
    return _lib


def ptr(x) -> int | None:
    """Device or host address of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _check(rc: int, where: str, ctx) -> None:
    if rc != AG_OK:
        msg = lib().ag_last_error(ctx)
        raise AgError(rc, where, msg.decode() if msg else "")


def ag_abi_version() -> int:
    return lib().ag_abi_version()


def ag_config_default() -> ag_config:
    c = ag_config()
    lib().ag_config_default(ctypes.byref(c))
    return c


def ag_create(cfg: ag_config, stream: int | None = None) -> int:
    out = _vp()
    rc = lib().ag_create(ctypes.byref(cfg), stream, ctypes.byref(out))
    _check(rc, "ag_create", None)
    return out.value


def ag_destroy(ctx: int) -> None:
    _check(lib().ag_destroy(ctx), "ag_destroy", ctx)


def ag_set_commands(ctx: int, modes, targets) -> None:
    _check(lib().ag_set_commands(ctx, ptr(modes), ptr(targets)), "ag_set_commands", ctx)


def ag_set_obstacles(ctx: int, boxes) -> None:
    _check(lib().ag_set_obstacles(ctx, ptr(boxes)), "ag_set_obstacles", ctx)


def ag_set_body(ctx: int, body) -> None:
    _check(lib().ag_set_body(ctx, ptr(body)), "ag_set_body", ctx)


def ag_get_obstacles(ctx: int, boxes) -> None:
    _check(lib().ag_get_obstacles(ctx, ptr(boxes)), "ag_get_obstacles", ctx)


def ag_render_depth(ctx: int, width: int, height: int, hfov: float, max_range: float, cam_offset, env_ids,
                    n_cams: int, depth) -> None:
    off = None if cam_offset is None else (ctypes.c_float * 3)(*cam_offset)
    rc = lib().ag_render_depth(ctx, int(width), int(height), float(hfov), float(max_range),
                               ctypes.byref(off) if off is not None else None, ptr(env_ids), int(n_cams), ptr(depth))
    _check(rc, "ag_render_depth", ctx)


def ag_collision_tests_run(ctx: int) -> int:
    """Collision tests the last ag_step ran (include/ag_measure.h)."""
    out = ctypes.c_uint64()
    _check(lib().ag_collision_tests_run(ctx, ctypes.byref(out)), "ag_collision_tests_run", ctx)
    return int(out.value)


def ag_render_depth_ieee(ctx: int, width: int, height: int, hfov: float, max_range: float, cam_offset, env_ids,
                         n_cams: int, depth) -> None:
    """ag_render_depth with correctly rounded reciprocals (include/ag_measure.h)."""
    off = None if cam_offset is None else (ctypes.c_float * 3)(*cam_offset)
    rc = lib().ag_render_depth_ieee(ctx, int(width), int(height), float(hfov), float(max_range),
                                    ctypes.byref(off) if off is not None else None, ptr(env_ids), int(n_cams),
                                    ptr(depth))
    _check(rc, "ag_render_depth_ieee", ctx)


def ag_depth_live_pairs(ctx: int, width: int, height: int, hfov: float, max_range: float, cam_offset, env_ids,
                        n_cams: int) -> int:
    """(pixel, box) pairs ag_render_depth tests after culling (include/ag_measure.h)."""
    off = None if cam_offset is None else (ctypes.c_float * 3)(*cam_offset)
    out = ctypes.c_uint64()
    rc = lib().ag_depth_live_pairs(ctx, int(width), int(height), float(hfov), float(max_range),
                                   ctypes.byref(off) if off is not None else None, ptr(env_ids), int(n_cams),
                                   ctypes.byref(out))
    _check(rc, "ag_depth_live_pairs", ctx)
    return int(out.value)


def ag_set_obstacle_randomization(ctx: int, env_min, env_max, per_box) -> None:
    """per_box: a sequence of ag_box_randomization (one per obstacle) or None to disable."""
    lo = (ctypes.c_float * 3)(*env_min) if env_min is not None else None
    hi = (ctypes.c_float * 3)(*env_max) if env_max is not None else None
    arr = None if per_box is None else (ag_box_randomization * len(per_box))(*per_box)
    rc = lib().ag_set_obstacle_randomization(ctx, ctypes.byref(lo) if lo else None, ctypes.byref(hi) if hi else None,
                                             ctypes.cast(arr, ctypes.c_void_p) if arr is not None else None)
    _check(rc, "ag_set_obstacle_randomization", ctx)


def box_randomization(pos_min=(0, 0, 0), pos_max=(1, 1, 1), euler_min=(0, 0, 0), euler_max=(0, 0, 0), lock=0,
                      fixed=(0, 0, 0, 0, 0, 0)) -> ag_box_randomization:
    r = ag_box_randomization()
    r.pos_min[:], r.pos_max[:] = list(pos_min), list(pos_max)
    r.euler_min[:], r.euler_max[:] = list(euler_min), list(euler_max)
    r.lock = lock
    r.fixed[:] = list(fixed)
    return r


def ag_step(ctx: int, n_substeps: int) -> None:
    _check(lib().ag_step(ctx, int(n_substeps)), "ag_step", ctx)


def ag_step_plain(ctx: int, n_substeps: int) -> None:
    _check(lib().ag_step_plain(ctx, int(n_substeps)), "ag_step_plain", ctx)


def ag_inject_failure(ctx: int, why: str | None = None) -> None:
    _check(lib().ag_inject_failure(ctx, why.encode() if why else None), "ag_inject_failure", ctx)


def ag_measure_fp32_peak(stream: int = 0, iters: int = 10000, reps: int = 5, out=None) -> dict:
    """FP32 FMA-chain throughput of the current device (include/ag_measure.h).
    `out` may be given to receive the raw struct (used to pass NULL in tests)."""
    r = ag_fp32_peak()
    rc = lib().ag_measure_fp32_peak(stream or None, iters, reps, ctypes.byref(r) if out is None else out)
    _check(rc, "ag_measure_fp32_peak", None)
    return {k: getattr(r, k) for k, _ in ag_fp32_peak._fields_}


def ag_query_alu_peak(device: int = 0) -> dict:
    """Derived FP32 CUDA-core peak of a device from its own attributes
    (include/ag_measure.h)."""
    r = ag_alu_peak()
    _check(lib().ag_query_alu_peak(int(device), ctypes.byref(r)), "ag_query_alu_peak", None)
    return {k: getattr(r, k) for k, _ in ag_alu_peak._fields_}


def ag_eval_controller(ctx: int, state, wrench) -> None:
    _check(lib().ag_eval_controller(ctx, ptr(state), ptr(wrench)), "ag_eval_controller", ctx)


def ag_reset(ctx: int, mask, seed: int) -> None:
    _check(lib().ag_reset(ctx, ptr(mask), int(seed) & (2**64 - 1)), "ag_reset", ctx)


def ag_get_state(ctx: int, state=None, collided=None, reset_ids=None, want_count: bool = False) -> int | None:
    cnt = ctypes.c_uint32(0)
    rc = lib().ag_get_state(ctx, ptr(state), ptr(collided), ptr(reset_ids), ctypes.byref(cnt) if want_count else None)
    _check(rc, "ag_get_state", ctx)
    return cnt.value if want_count else None


def ag_get_motors(ctx: int, motors=None, epoch=None) -> None:
    _check(lib().ag_get_motors(ctx, ptr(motors), ptr(epoch)), "ag_get_motors", ctx)


def ag_set_state(ctx: int, state, motors=None, epoch=None) -> None:
    _check(lib().ag_set_state(ctx, ptr(state), ptr(motors), ptr(epoch)), "ag_set_state", ctx)


def ag_synchronize(ctx: int) -> None:
    _check(lib().ag_synchronize(ctx), "ag_synchronize", ctx)


def ag_get_config(ctx: int) -> ag_config:
    c = ag_config()
    _check(lib().ag_get_config(ctx, ctypes.byref(c)), "ag_get_config", ctx)
    return c


def ag_set_gains(ctx: int, gains12) -> None:
    _check(lib().ag_set_gains(ctx, ptr(gains12)), "ag_set_gains", ctx)


def ag_rollout_loss(ctx: int, n_steps: int, w_pos: float, w_omega: float, p_goal, loss, saturated=None) -> None:
    _check(lib().ag_rollout_loss(ctx, int(n_steps), float(w_pos), float(w_omega), ptr(p_goal), ptr(loss),
                                 ptr(saturated)), "ag_rollout_loss", ctx)


def ag_backward(ctx: int, loss_weights=None, grad_x0=None, grad_gains=None, grad_gains_per_env=None,
                grad_targets=None) -> None:
    _check(lib().ag_backward(ctx, ptr(loss_weights), ptr(grad_x0), ptr(grad_gains), ptr(grad_gains_per_env),
                             ptr(grad_targets)), "ag_backward", ctx)


def ag_reach_config_default() -> ag_reach_config:
    c = ag_reach_config()
    lib().ag_reach_config_default(ctypes.byref(c))
    return c


def ag_reach_begin(ctx: int, cfg: ag_reach_config, goals) -> None:
    _check(lib().ag_reach_begin(ctx, ctypes.byref(cfg), ptr(goals)), "ag_reach_begin", ctx)


def ag_reach_step(ctx: int, actions, obs, reward, done) -> None:
    _check(lib().ag_reach_step(ctx, ptr(actions), ptr(obs), ptr(reward), ptr(done)), "ag_reach_step", ctx)


def ag_reach_observe(ctx: int, obs) -> None:
    _check(lib().ag_reach_observe(ctx, ptr(obs)), "ag_reach_observe", ctx)


def ag_server_config_default() -> ag_server_config:
    c = ag_server_config()
    lib().ag_server_config_default(ctypes.byref(c))
    return c


def ag_server_create(cfg: ag_server_config) -> int:
    out = _vp()
    rc = lib().ag_server_create(ctypes.byref(cfg), ctypes.byref(out))
    if rc != AG_OK:
        raise AgError(rc, "ag_server_create", "")
    return out.value


def ag_server_submit(server: int, req: ag_request) -> int:
    rid = ctypes.c_uint64()
    rc = lib().ag_server_submit(server, ctypes.byref(req), ctypes.byref(rid))
    if rc != AG_OK:
        raise AgError(rc, "ag_server_submit", "")
    return rid.value


def ag_server_wait(server: int, rid: int, timeout_s: float, final_state=None, epoch=None) -> float:
    """Returns the request's latency in ms (final_state / epoch: host arrays or None)."""
    lat = ctypes.c_double()
    rc = lib().ag_server_wait(server, int(rid), float(timeout_s), ptr(final_state), ptr(epoch), ctypes.byref(lat))
    if rc != AG_OK:
        raise AgError(rc, "ag_server_wait", "")
    return lat.value


def ag_server_get_stats(server: int) -> ag_server_stats:
    st = ag_server_stats()
    rc = lib().ag_server_get_stats(server, ctypes.byref(st))
    if rc not in (AG_OK, AG_ERR_STATE):
        raise AgError(rc, "ag_server_get_stats", "")
    return st


def ag_server_destroy(server: int) -> None:
    lib().ag_server_destroy(server)


def ag_last_error(ctx: int | None) -> str:
    m = lib().ag_last_error(ctx)
    return m.decode() if m else ""


AG_NOALLOC_MAX_ENVS = 65536


def ag_step_plain_noalloc(cfg: ag_config, stream, n_substeps: int, seed: int, state, motors, body, modes, targets,
                          boxes, epoch, collided, reset_ids, n_reset) -> None:
    """Context-free unfused step that allocates no device memory (all buffers
    are the caller's device buffers; see include/ag.h)."""
    err = ctypes.create_string_buffer(256)
    rc = lib().ag_step_plain_noalloc(ctypes.byref(cfg), stream, int(n_substeps), int(seed) & (2**64 - 1),
                                     ptr(state), ptr(motors), ptr(body), ptr(modes), ptr(targets), ptr(boxes),
                                     ptr(epoch), ptr(collided), ptr(reset_ids), ptr(n_reset), err, len(err))
    if rc != AG_OK:
        raise AgError(rc, "ag_step_plain_noalloc", err.value.decode())
