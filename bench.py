"""Fleet-step throughput bench: vehicle-steps/s of the fused kernel vs the
unfused one-launch-per-stage path, on 1,048,576 quadrotors with mixed command
modes, RK4 (4 substeps of 2.5 ms per 10 ms step) and 16 oriented boxes each.

One bench step = one ag_step call that advances the whole fleet by
STEPS_PER_CALL simulated steps (all stages: controller, allocation, motor
lag, RK4, renormalisation, sphere-vs-box test, Philox resets, compaction).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--envs N_ENVS] [--steps-per-call C] [--parts fused,plain,e2e,paper,mixed,depth,task,adjoint,serve]

--envs / --steps-per-call / --parts run a reduced case of the same workload
(for profiler captures); the default is the full workload and every part.

Under torchrun each rank runs an independent replica on its own GPU (the
environments are independent; there is no exchange step). Rank 0 prints one
JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "vehicle-steps/s at 1M quads (fused vs plain step); serving p50/p99 ms"
UNIT = "vehicle-steps/s"
STEPS_PER_CALL = 1000          # the obstacle workload's horizon: one call = one full rollout
WORKLOAD = "obstacles"
WORKLOAD_TEXT = ("1,048,576 quadrotors; command mode uniform over position / body velocity / attitude+thrust; "
                 "RK4, 4 substeps x 2.5 ms per 10 ms step; 16 random oriented boxes per env "
                 "(half-extents U[0.1,1] m, centres U[-5,5]^3 m); r = 0.2 m sphere; collision -> Philox reset; "
                 f"{STEPS_PER_CALL} steps per call")
# Algorithmic FP32 operations per vehicle-step of this workload: the FP64
# oracle run with an operation-counting scalar (adds, muls, divs, square
# roots, transcendentals; comparisons excluded), averaged over the three
# command modes, RK4 x 4 substeps + 16 boxes. tests/test_bench_constants.py
# re-derives it.
FLOP_PER_VEHICLE_STEP = 4588.0
# Of which one sphere-vs-box test, per box (40 multiplications, 26 additions;
# pinned by a hand count in tests/test_oracle_pins.py). The fused step skips
# tests that provably cannot hit; the work it performs is counted with
# ag_collision_tests_run.
FLOP_PER_BOX_TEST = 66.0
# The same count for the other lines: the mixed fleet (body velocity, SIE,
# drag, 40 % quad / 40 % hexa / 20 % octo) and the paper shape (attitude and
# body velocity, SIE, quads, no boxes).
FLOP_PER_VEHICLE_STEP_MIXED = 584.4
# Bytes the unfused path moves per vehicle-step of the bench workload: per
# substep the controller (state 52, mode 1, targets 16, body 16 in; command
# 16 out), allocation (command 16, motors 16 in; motors 16, wrench 16 out)
# and integrator (state 52, wrench 16, body 16 in; state 52 out), 301 B x 4;
# per step the collision test (position 12, 16 boxes x 40 in; hit byte out)
# and the reset pass (hit byte in).
PLAIN_BYTES_PER_VEHICLE_STEP = 301 * 4 + 12 + 16 * 40 + 1 + 1
HBM_PEAK_GBS = 6788.3  # measured GB300 copy bandwidth (MEASURED_PEAKS.json, hbm_gbs)


def hbm_peak_gbs() -> float:
    """The machine's measured copy bandwidth (MEASURED_PEAKS.json when present,
    else the figure it held when these lines were written)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return HBM_PEAK_GBS


FLOP_PER_VEHICLE_STEP_PAPER_SHAPE = 528.5


def alu_peak_tflops(info: dict) -> float:
    """FP32 CUDA-core peak from a device's own attributes: SMs x FP32 lanes per
    SM x 2 FLOP per FMA x peak SM clock (ag_query_alu_peak)."""
    return info["sm_count"] * info["fp32_lanes_per_sm"] * 2 * info["max_sm_clock_khz"] * 1e3 / 1e12


# Algorithmic bytes of one fused launch per vehicle: state in+out (13 f32 x 2),
# motors in+out (4 x 2), body (4), targets (4), mode (1 B), epoch in+out (2 x 4),
# boxes (16 x 10 f32), collided flag (1 B), reset-list entry (4 B, upper bound)
BYTES_PER_VEHICLE_LAUNCH = 4 * (26 + 8 + 4 + 4) + 1 + 8 + 4 * 160 + 1 + 4
# DRAM traffic of one full-size fused launch (1,048,576 envs, 1,000 steps):
# dram__bytes_read.sum + dram__bytes_write.sum from a one-pass ncu capture of
# exactly this launch (797.11 MB + 68.19 MB). It scales with the fleet size
# (each env is loaded and stored once per launch; the rare collision tests
# after the first re-read a few boxes), not with the step count.
TRAFFIC_BYTES_FULL_LAUNCH = 797.112064e6 + 68.190976e6
# Algorithmic bytes of one reach-task step per quad: read action 16, goal 12,
# step counter 4, state 52, motors 16, body 16, epoch 4, mode 1 (121 B);
# written state 52, motors 16, epoch 4, collided flag 1, command 16,
# reward 4, done 1, step counter 4, observation 52 (150 B).
TASK_BYTES_PER_ENV_STEP = (16 + 12 + 4 + 52 + 16 + 16 + 4 + 1) + (52 + 16 + 4 + 1 + 16 + 4 + 1 + 4 + 52)
# Algorithmic bytes of one depth frame: the float32 270 x 480 image written
# (the boxes and poses read are under 1 KB per camera).
DEPTH_BYTES_PER_FRAME = 270 * 480 * 4
# Algorithmic FP32 operations of the depth caster (the oracle's ray_box_depth
# run with the operation-counting scalar, comparisons excluded), by what each
# part repeats over: per pixel (its ray R d_c), per (camera, box) pair (R_b^T
# and the camera origin in the box frame), per (pixel, box) pair (the ray in
# the box frame and the slab intervals). tests/test_bench_constants.py
# re-derives them.
DEPTH_FLOP_PER_PIXEL, DEPTH_FLOP_PER_CAMERA_BOX, DEPTH_FLOP_PER_PIXEL_BOX = 21.0, 57.0, 27.0
# Algorithmic operations of one step of the differentiable rollout (position
# mode, quadrotor, SIE, one substep, the step's loss term): the forward step
# and its reverse-mode adjoint (the oracle run with the reverse-counting
# scalar, every elementary operation's adjoint rule counted). The backward
# launch's algorithmic work per vehicle-step is one forward recomputation
# from the checkpoints plus the adjoint.
FLOP_PER_VEHICLE_STEP_ADJ_FWD = 460.0
FLOP_PER_VEHICLE_STEP_ADJ_REV = 1217.0


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.lines: list[str] = []
        self.proc = None
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- GPU arm ----
def make_fleet(w, inp, seed):
    from paper_2305_16510_gb300.fleet import Fleet
    fl = Fleet(w.n_envs, substeps_per_step=w.substeps_per_step, integrator=w.integrator, n_obstacles=w.n_obstacles,
               n_hexa=w.n_hexa, n_octo=w.n_octo, dt=w.dt, motor_tau=w.motor_tau, drag=w.drag, seed=seed)
    fl.set_body(inp.body)
    fl.set_commands(inp.modes, inp.targets)
    if inp.boxes is not None:
        fl.set_obstacles(inp.boxes)
    fl.reset(None, seed)
    return fl


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """The largest x of all ranks (the slowest rank's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, slowest_secs: float) -> float:
    """Weak scaling: every rank processes units_per_rank in its own fleet; the
    job's rate is all ranks' units over the slowest rank's time."""
    return units_per_rank * world / slowest_secs


def time_calls(fl, call, k: int, world: int):
    """Times k calls with CUDA events on the fleet's stream; returns
    (total seconds across ranks, per-call event durations in ms)."""
    import torch
    stream = fl.stream
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for a, b in evs:
        a.record(stream)
        call()
        b.record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    total_ms = t0.elapsed_time(t1)
    per = [a.elapsed_time(b) for a, b in evs]
    return max_over_ranks(total_ms / 1e3, world), per


def rate_stats(units_per_call: float, per_ms: list[float]) -> dict:
    """Median and range of per-call rates (units per call over each call's
    CUDA-event duration)."""
    rates = sorted(units_per_call / (ms * 1e-3) for ms in per_ms)
    return {"median": float(np.median(rates)), "range": [rates[0], rates[-1]]}


def gpu_arm(args) -> dict | None:
    import torch
    from paper_2305_16510_gb300 import build, workloads as W
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    build.build()
    from paper_2305_16510_gb300 import _abi
    alu = _abi.ag_query_alu_peak(torch.cuda.current_device())
    alu_peak = alu_peak_tflops(alu)
    w = W.WORKLOADS[WORKLOAD]
    if args.envs:
        w = W.scaled(w, args.envs)
    C = args.steps_per_call
    parts = set(args.parts.split(","))
    seed = args.seed + rank
    inp = W.make_inputs(w, seed)
    fl = make_fleet(w, inp, seed)
    n_sub = C * w.substeps_per_step

    # ---- fused (headline)
    for _ in range(args.warmup):
        fl.step(C)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        secs, per = time_calls(fl, lambda: fl.step(C), args.steps, world)
    value = whole_job_rate(w.n_envs * C * args.steps, world, secs)
    ms_per_step = secs * 1e3 / args.steps
    launch_ms = float(np.mean(per))
    achieved_tflops = w.n_envs * C * FLOP_PER_VEHICLE_STEP / (launch_ms * 1e-3) / 1e12
    _, n_reset = fl.events()
    # collision tests the last timed call ran, of the n_envs x C the method specifies
    tests_frac = _abi.ag_collision_tests_run(fl.ctx) / float(w.n_envs * C)
    flop_performed = FLOP_PER_VEHICLE_STEP - w.n_obstacles * FLOP_PER_BOX_TEST * (1.0 - tests_frac)
    out = {}
    # check of the derived ALU peak: an FMA-chain kernel of the library, run
    # after the timed region on the same stream (about 0.2 s)
    fma_chain = _abi.ag_measure_fp32_peak(fl.stream.cuda_stream, iters=10000, reps=5)

    # ---- unfused comparison path (same fleet, same call size)
    if "plain" in parts:
        k_plain = max(1, min(args.steps, 3))
        fl.step_plain(C)
        torch.cuda.synchronize()
        secs_p, per_p = time_calls(fl, lambda: fl.step_plain(C), k_plain, world)
        plain_value = w.n_envs * C * k_plain * world / secs_p
        out["plain"] = {"value": plain_value, "unit": UNIT, "ms_per_step": secs_p * 1e3 / k_plain,
                        "bytes_per_vehicle_step": PLAIN_BYTES_PER_VEHICLE_STEP,
                        "hbm_frac": plain_value / world * PLAIN_BYTES_PER_VEHICLE_STEP / 1e9 / hbm_peak_gbs(),
                        "launches_per_step": C * (3 * w.substeps_per_step + 2) + 1,
                        "fused_over_plain": value / plain_value, **rate_stats(w.n_envs * C, per_p)}

    # ---- end to end through the C-ABI with host buffers: per call, upload the
    # commands from pinned host memory, step, read the state back
    modes_h = torch.from_numpy(inp.modes).pin_memory()
    targets_h = torch.from_numpy(inp.targets).pin_memory()
    state_h = torch.empty((13, w.n_envs), dtype=torch.float32).pin_memory()

    def e2e_call():
        _abi.ag_set_commands(fl.ctx, modes_h, targets_h)
        _abi.ag_step(fl.ctx, n_sub)
        _abi.ag_get_state(fl.ctx, state=state_h)

    if "e2e" in parts:
        e2e_call()
        fl.synchronize()
        k_e2e = max(1, min(args.steps, 5))
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            e2e_call()
            fl.synchronize()
        e2e_secs = max_over_ranks(time.perf_counter() - t0, world)
        e2e_value = w.n_envs * C * k_e2e * world / e2e_secs
        h2d = inp.modes.nbytes + inp.targets.nbytes
        d2h = state_h.numel() * 4
        assert np.isfinite(state_h.numpy()).all()
        out["e2e"] = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h)}

    # ---- the paper's own throughput shape (context only)
    if "paper" in parts:
        ws = W.WORKLOADS["paper_shape"]
        inp_s = W.make_inputs(ws, seed)
        fs = make_fleet(ws, inp_s, seed)
        fs.step(100)
        torch.cuda.synchronize()
        k_s = 5
        secs_s, per_s = time_calls(fs, lambda: fs.step(1000), k_s, world)
        v_s = ws.n_envs * 1000 * k_s * world / secs_s
        st = rate_stats(ws.n_envs * 1000, per_s)
        out["paper_shape"] = {"value": v_s, "unit": UNIT,
                              "alu_frac": v_s / world * FLOP_PER_VEHICLE_STEP_PAPER_SHAPE / 1e12 / alu_peak,
                              **st,
                              "workload": "131,072 quads, attitude/body-velocity commands, no obstacles, SIE, "
                                          "1 substep",
                              "paper_value": 3.8e6,
                              "paper_hardware": "2x RTX 3090 + TR PRO 3975WX (Isaac Gym/PhysX)"}
        fs.close()
    fl.close()
    if "mixed" in parts:
        out["mixed"] = mixed_part(seed, world, alu_peak)
    if "depth" in parts:
        out["depth"] = depth_part(seed, world, alu_peak)
    if "task" in parts:
        out["task"] = task_part(seed, world)
    if "adjoint" in parts:
        out["adjoint"] = adjoint_part(seed, world, alu_peak)
    if "serve" in parts:
        out["serving"] = serving_part(seed)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank != 0:
        return None
    clocks = clk.summary()
    full_size = w.n_envs == 1 << 20 and C == STEPS_PER_CALL
    wtext = WORKLOAD_TEXT if full_size else f"reduced case of the same recipe: {w.n_envs} envs, {C} steps per call"
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded numpy commands and boxes; Philox initial states)",
        "config": {"workload": wtext, "n_envs": w.n_envs, "steps_per_call": C,
                   "substeps_per_step": w.substeps_per_step, "integrator": "rk4", "boxes_per_env": w.n_obstacles,
                   "l2": "no flush: inputs exceed L2 (boxes 671 MB + state 55 MB per call)",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": achieved_tflops / alu_peak,
                     "traffic": TRAFFIC_BYTES_FULL_LAUNCH if full_size else None,
                     "kernel": "k_fused_step<RK4, quad>", "launch_ms": launch_ms,
                     "flop_per_vehicle_step": FLOP_PER_VEHICLE_STEP,
                     # the same over the work the launch performed: every step's controller and
                     # integration, and only the collision tests it ran (tests_run of n_envs x steps)
                     "tests_run": tests_frac,
                     "frac_performed": w.n_envs * C * flop_performed / (launch_ms * 1e-3) / 1e12 / alu_peak,
                     "peak_source": (f"derived from the device: {alu['sm_count']} SM x {alu['fp32_lanes_per_sm']} "
                                     f"FP32 lanes x 2 x {alu['max_sm_clock_khz'] / 1e3:.0f} MHz "
                                     "(MEASURED_PEAKS has no FP32 figure)"),
                     "device": alu,
                     "fma_chain_check": {
                         "scalar_tflops": fma_chain["scalar_tflops"], "packed_tflops": fma_chain["packed_tflops"],
                         "frac_of_packed": achieved_tflops / fma_chain["packed_tflops"],
                         "what": "measured FMA-chain kernels (ag_measure_fp32_peak: scalar fmaf and packed "
                                 "__ffma2_rn, best of 5, grid = SMs x resident blocks), run after the timed region"},
                     "algorithmic_bytes_per_launch": BYTES_PER_VEHICLE_LAUNCH * w.n_envs},
        "gpu_launches": args.steps,
        "clocks": clocks,
        "resets_last_call": int(n_reset.numel()),
        **rate_stats(w.n_envs * C, per),
    }
    res.update(out)
    return res


# ------------------------------------------------------------- mixed fleet --
def mixed_part(seed: int, world: int, alu_peak: float) -> dict:
    """4,194,304 vehicles (40 % quad, 40 % hexa, 20 % octo), randomised mass
    and inertia, motor lag, drag, body-velocity commands, semi-implicit Euler:
    the 500-step rollout as 10 calls of 50 steps, each followed by a 1 %
    Bernoulli ag_reset mask (masks pre-generated on the device)."""
    import torch
    from paper_2305_16510_gb300 import workloads as W
    w = W.WORKLOADS["mixed"]
    inp = W.make_inputs(w, seed)
    fl = make_fleet(w, inp, seed)
    rng = np.random.default_rng(seed + 100)
    masks = [torch.from_numpy(W.reset_mask(w.n_envs, w.reset_prob, rng)).cuda() for _ in range(10)]
    from paper_2305_16510_gb300 import _abi

    def rollout():
        for k in range(10):
            fl.step(w.reset_every)
            _abi.ag_reset(fl.ctx, masks[k], seed + k)

    rollout()
    torch.cuda.synchronize()
    k = 5
    secs, per = time_calls(fl, rollout, k, world)
    fl.close()
    v = w.n_envs * 500 * k * world / secs
    st = rate_stats(w.n_envs * 500, per)
    return {"value": v, "unit": UNIT, "ms_per_rollout": secs * 1e3 / k,
            "alu_frac": v / world * FLOP_PER_VEHICLE_STEP_MIXED / 1e12 / alu_peak, **st,
            "workload": "4,194,304 vehicles (1,677,722 quad / 1,677,722 hexa / 838,860 octo), mass and inertia "
                        "x U[0.8, 1.2], tau 0.03, drag 0.1, body-velocity targets U[-2, 2]^3, SIE, 500 steps "
                        "as 10 x (50-step ag_step + 1 % ag_reset mask)"}


# ------------------------------------------------------------------- depth --
def depth_part(seed: int, world: int, alu_peak: float) -> dict:
    """2^10 robots, each a 270 x 480 depth camera (87 deg horizontal field of
    view, 10 m range) ray-cast against its environment's 16 boxes."""
    import math
    import torch
    from paper_2305_16510_gb300 import _abi, workloads as W
    w = W.scaled(W.WORKLOADS[WORKLOAD], 1024)
    inp = W.make_inputs(w, seed)
    fl = make_fleet(w, inp, seed)
    fl.step(10)
    H, Wd, hfov, rng_max = 270, 480, math.radians(87), 10.0
    out = torch.empty((1024, H, Wd), dtype=torch.float32, device="cuda")

    def render():
        fl.render_depth(Wd, H, hfov, rng_max, out=out)

    for _ in range(3):
        render()
    torch.cuda.synchronize()
    k = 20
    secs, per = time_calls(fl, render, k, world)
    # pixel-box pairs the kernel tests after its conservative culling
    live = _abi.ag_depth_live_pairs(fl.ctx, Wd, H, hfov, rng_max, None, None, 1024)
    fl.close()
    frames = 1024 * k * world
    launch_s = float(np.mean(per)) * 1e-3
    all_pairs = 1024 * H * Wd * w.n_obstacles
    per_launch = 1024 * (H * Wd * DEPTH_FLOP_PER_PIXEL + w.n_obstacles * DEPTH_FLOP_PER_CAMERA_BOX)
    return {"value": frames / secs, "unit": "depth frames/s", "ms_per_1024_frames": float(np.mean(per)),
            **rate_stats(1024, per),
            "pixel_box_pairs_per_s": frames * H * Wd * w.n_obstacles / secs,  # culled pairs included
            "live_pair_frac": live / all_pairs,
            "flop": {"per_pixel": DEPTH_FLOP_PER_PIXEL, "per_camera_box": DEPTH_FLOP_PER_CAMERA_BOX,
                     "per_pixel_box": DEPTH_FLOP_PER_PIXEL_BOX},
            # the method's work that the kernel performs: every pixel's ray, every camera-box setup
            # and every live pair's slab test (comparisons and min/max are not counted)
            "alu_frac": (per_launch + live * DEPTH_FLOP_PER_PIXEL_BOX) / launch_s / 1e12 / alu_peak,
            # the same with every pair counted, as a test without culling would do (context)
            "alu_frac_all_pairs": (per_launch + all_pairs * DEPTH_FLOP_PER_PIXEL_BOX) / launch_s / 1e12 / alu_peak,
            "hbm_frac": 1024 * DEPTH_BYTES_PER_FRAME / launch_s / 1e9 / hbm_peak_gbs(),
            "bound": "instruction issue (slab min/max on the ALU pipe, reciprocals on XU) above the HBM write "
                     "floor of the image",
            "workload": "1,024 robots x 270 x 480 depth camera, 16 oriented boxes per environment, 87 deg hfov",
            "paper_value": 1800.0, "paper_hardware": "2x RTX 3090, Isaac Gym camera sensors (graphics renderer)"}


# -------------------------------------------------------------------- task --
def task_part(seed: int, world: int) -> dict:
    """Reach-a-setpoint task steps (ag_reach_step: actions to attitude
    commands, one fleet step, reward, termination, auto-reset, observations)
    over 1,048,576 quads, semi-implicit Euler, 1 substep, no obstacles; also
    with 50 steps captured in a CUDA graph and replayed."""
    import torch
    from paper_2305_16510_gb300 import _abi
    from paper_2305_16510_gb300.task import ReachEnv
    n = 1 << 20
    rng = np.random.default_rng(seed)
    goals = torch.from_numpy(rng.uniform(-1.0, 1.0, (3, n)).astype(np.float32))
    side = torch.cuda.Stream()          # graph capture needs a stream other than the legacy default one
    with torch.cuda.stream(side):
        env = ReachEnv(n, goals=goals, seed=seed, stream=side)
        env.reset()
        actions = torch.from_numpy(rng.uniform(-0.3, 0.3, (n, 4)).astype(np.float32)).cuda()
    torch.cuda.synchronize()

    def step():
        _abi.ag_reach_step(env.fleet.ctx, actions, env.obs, env.reward, env.done)

    for _ in range(5):
        step()
    torch.cuda.synchronize()
    k, per_graph = 200, 50
    secs, per = time_calls(env.fleet, step, k, world)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        for _ in range(per_graph):
            step()
    with torch.cuda.stream(side):
        g.replay()
        torch.cuda.synchronize()
        secs_g, per_g = time_calls(env.fleet, g.replay, k // per_graph, world)
    env.close()
    return {"value": n * k * world / secs, "unit": "task env-steps/s", "ms_per_step": float(np.mean(per)),
            **rate_stats(n, per),
            "bytes_per_env_step": TASK_BYTES_PER_ENV_STEP,
            # algorithmic bytes of one launch over its mean CUDA-event duration
            "hbm_frac": n * TASK_BYTES_PER_ENV_STEP / (float(np.mean(per)) * 1e-3) / 1e9 / hbm_peak_gbs(),
            "workload": "reach-a-setpoint, 1,048,576 quads, attitude interface, SIE 1 substep, no obstacles, "
                        "obs [n,13] + reward + done per step", "launches_per_step": 1,
            "cuda_graph": {"value": n * k * world / secs_g, "ms_per_step": secs_g * 1e3 / k,
                           "steps_per_graph": per_graph, **rate_stats(n * per_graph, per_g)}}


# ----------------------------------------------------------------- adjoint --
def adjoint_part(seed: int, world: int, alu_peak: float) -> dict:
    """Differentiable rollout at 65,536 quads x 256 steps (position mode, SIE,
    checkpoint every 32): recorded forward + hand-written adjoint. Each half
    is timed with CUDA events on the fleet's stream."""
    import torch
    from paper_2305_16510_gb300 import _abi, workloads as W
    w = W.WORKLOADS["adjoint"]
    inp = W.make_inputs(w, seed)
    fl = make_fleet(w, inp, seed)
    n, H = w.n_envs, w.horizon
    goal = torch.from_numpy(np.ascontiguousarray(inp.targets[0:3])).cuda()
    loss = torch.empty(n, device="cuda")
    gx = torch.empty((13, n), device="cuda")
    gg = torch.empty(12, device="cuda")
    x0, m0 = fl.state().clone(), fl.motors().clone()
    stream = fl.stream

    def fwd_bwd(ev=None):
        fl.set_state(x0, m0)
        if ev:
            ev[0].record(stream)
        _abi.ag_rollout_loss(fl.ctx, H, 1.0, 0.01, goal, loss)
        if ev:
            ev[1].record(stream)
        _abi.ag_backward(fl.ctx, None, gx, gg, None)
        if ev:
            ev[2].record(stream)

    for _ in range(3):
        fwd_bwd()
    torch.cuda.synchronize()
    k = 20
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(k)]
    barrier(world)
    t0 = time.perf_counter()
    for e in evs:
        fwd_bwd(e)
    torch.cuda.synchronize()
    secs = max_over_ranks(time.perf_counter() - t0, world)
    fl.close()
    fwd_ms = [e[0].elapsed_time(e[1]) for e in evs]
    bwd_ms = [e[1].elapsed_time(e[2]) for e in evs]
    units = n * H
    fwd_s, bwd_s = float(np.median(fwd_ms)) * 1e-3, float(np.median(bwd_ms)) * 1e-3
    return {"value": units * k * world / secs, "unit": "vehicle-steps/s (forward + adjoint)",
            "ms_per_rollout": secs * 1e3 / k, **rate_stats(units, [a + b for a, b in zip(fwd_ms, bwd_ms)]),
            "record_ms": fwd_s * 1e3, "backward_ms": bwd_s * 1e3,
            "flop_per_vehicle_step": {"forward": FLOP_PER_VEHICLE_STEP_ADJ_FWD,
                                      "reverse": FLOP_PER_VEHICLE_STEP_ADJ_FWD + FLOP_PER_VEHICLE_STEP_ADJ_REV},
            "alu_frac_record": units * FLOP_PER_VEHICLE_STEP_ADJ_FWD / fwd_s / 1e12 / alu_peak,
            "alu_frac_backward": units * (FLOP_PER_VEHICLE_STEP_ADJ_FWD + FLOP_PER_VEHICLE_STEP_ADJ_REV)
            / bwd_s / 1e12 / alu_peak,
            "workload": "65,536 quads, position mode, SIE, horizon 256, checkpoint every 32 steps, "
                        "gradients w.r.t. x0 (13/vehicle) and 12 gains"}


# ----------------------------------------------------------------- serving --
SERVE_LAMBDA = 200.0           # requests per second (Poisson arrivals)
SERVE_REQUESTS = 2200          # 200 warm-up + 2,000 measured
SERVE_WARMUP = 200
SERVE_REPLAYS = 3              # replays of the lambda = 200 trace (median and range of p99)
SERVE_POOL = 1 << 19           # pool of environments requests take slices of
SERVE_BUDGET = 40 << 30
# Capacity: the highest arrival rate of a sweep at which a policy keeps up
# with the offered load (completed work >= 95 % of the offered work rate) with
# p99 latency at or below SERVE_P99_BOUND_MS. The largest request of the trace
# (262,144 quads x 2,000 steps) needs about 94 ms of the whole GPU alone.
SERVE_P99_BOUND_MS = 250.0
# Rates of the sweep (requests/s) per policy; the highest of each overloads it,
# so the throughput there is that policy's ceiling.
SERVE_SWEEP = {"batched": (250.0, 300.0, 350.0, 400.0, 600.0),
               "one_per_launch": (150.0, 250.0, 300.0, 400.0)}
SERVE_SWEEP_SECONDS = 4.0      # arrivals per rate of the sweep: about this long, 200 .. 1,600 requests


def sweep_requests(lam: float) -> int:
    return int(min(1600, max(200, lam * SERVE_SWEEP_SECONDS)))


def serve_trace(n_req: int, seed: int = 7, lam: float = SERVE_LAMBDA, pool: int = 0):
    """Seeded request trace: exponential inter-arrivals at rate lam, fleet
    log-uniform in [256, 262144], horizon uniform in {50..2000}, obstacles from
    {0, 8, 32}. With pool > 0 the requests are the first n_req of a fixed
    sequence of `pool` drawn at unit rate, so traces at different rates hold
    the same requests and differ only in the time scale."""
    m = pool if pool else n_req
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0, size=m))[:n_req] / lam
    n = np.floor(np.exp(rng.uniform(np.log(256), np.log(262144), size=m))).astype(int)[:n_req]
    h = rng.integers(50, 2001, size=m)[:n_req]
    obs = rng.choice([0, 8, 32], size=m)[:n_req]
    off = (rng.uniform(size=m)[:n_req] * (SERVE_POOL - n)).astype(int)
    return [dict(t=float(t[i]), n=int(n[i]), h=int(h[i]), obs=int(obs[i]), off=int(off[i]), seed=1000 + i)
            for i in range(n_req)]


def run_trace(server, pool, trace, warm: int, cap_s: float) -> dict:
    """Replays the trace in real time against one server; returns latency and
    throughput of the requests after the warm-up that completed within cap_s."""
    t0 = time.perf_counter() + 0.2
    ids = [None] * len(trace)
    stop = threading.Event()

    def submitter():
        for i, r in enumerate(trace):
            delay = t0 + r["t"] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            if stop.is_set() or time.perf_counter() - t0 > cap_s:
                break
            ids[i] = server.submit(pool.request(r["n"], r["h"], r["obs"], r["seed"], r["off"]))

    th = threading.Thread(target=submitter, daemon=True)
    th.start()
    lat, done_at = {}, {}
    for i in range(len(trace)):
        while ids[i] is None and th.is_alive():
            time.sleep(0.0002)
        if ids[i] is None:
            break
        left = cap_s - (time.perf_counter() - t0)
        if left <= 0:
            break
        try:
            _, _, l = server.wait(ids[i], timeout_s=left, want_state=False)
        except Exception:
            break
        lat[i] = l
        done_at[i] = time.perf_counter() - t0
    stop.set()
    th.join()
    meas = [i for i in range(warm, len(trace)) if i in lat]
    submitted = sum(1 for x in ids if x is not None)
    if not meas:
        return {"completed": 0, "submitted": submitted}
    t_begin = trace[warm]["t"]
    t_end = max(done_at[i] for i in meas)
    work = sum(trace[i]["n"] * trace[i]["h"] for i in meas)
    offered = sum(trace[i]["n"] * trace[i]["h"] for i in range(warm, len(trace))) / \
        max(trace[-1]["t"] - t_begin, 1e-9)
    L = np.array([lat[i] for i in meas])
    edges = [0, 5, 10, 20, 50, 100, 200, 500, 1000, 2000, np.inf]
    counts, _ = np.histogram(L, bins=edges)
    return {"value": work / (t_end - t_begin), "unit": UNIT, "p50_ms": float(np.percentile(L, 50)),
            "p99_ms": float(np.percentile(L, 99)), "mean_ms": float(L.mean()), "completed": len(meas),
            "measured_of": len(trace) - warm, "submitted": submitted, "window_s": t_end - t_begin,
            "offered": offered,
            "latency_ms": {"p10": float(np.percentile(L, 10)), "p25": float(np.percentile(L, 25)),
                           "p75": float(np.percentile(L, 75)), "p90": float(np.percentile(L, 90)),
                           "max": float(L.max()),
                           "histogram": {f"{edges[k]}-{edges[k + 1]}": int(counts[k]) for k in range(len(counts))}}}


def keeps_up(r: dict) -> bool:
    """Every measured request completed, the completed work rate is at least
    95 % of the offered one, and p99 is within the bound."""
    return (r.get("completed", 0) == r.get("measured_of", -1) and r["value"] >= 0.95 * r["offered"]
            and r["p99_ms"] <= SERVE_P99_BOUND_MS)


def serving_part(seed: int) -> dict:
    from paper_2305_16510_gb300 import workloads as W
    from paper_2305_16510_gb300.serving import RequestPool, Server
    w = W.Workload("pool", SERVE_POOL, 4, 1, 32, SERVE_POOL, 0, 0,
                   mode_mix=(W.MODE_POSITION, W.MODE_BODY_VEL, W.MODE_ATT_THRUST))
    inp = W.make_inputs(w, seed)
    pool = RequestPool(inp.modes, inp.targets, inp.boxes.reshape(32 * 10, SERVE_POOL))
    del inp
    trace = serve_trace(SERVE_REQUESTS)
    out = {"workload": (f"Poisson {SERVE_LAMBDA:.0f} req/s, {SERVE_REQUESTS} requests ({SERVE_WARMUP} warm-up), "
                        "fleet log-uniform [256, 262144] quads, horizon U{50..2000} steps, modes mixed, "
                        "obstacles {0, 8, 32}, RK4 4 substeps, 40 GB budget, 50 steps per launch"),
           "offered_vehicle_steps_per_s": sum(r["n"] * r["h"] for r in trace) / trace[-1]["t"]}
    policies = {"batched": 1024, "one_per_launch": 1}
    with Server(max_active=policies["batched"], chunk_steps=50, hbm_budget_bytes=SERVE_BUDGET) as srv:
        runs = [run_trace(srv, pool, trace, SERVE_WARMUP, cap_s=120.0) for _ in range(SERVE_REPLAYS)]
        st = srv.stats()
    p99s = sorted(r["p99_ms"] for r in runs if r.get("completed"))
    mid = sorted(runs, key=lambda r: r.get("p99_ms", np.inf))[len(runs) // 2]   # the replay with the median p99
    out["batched"] = dict(mid)
    out["batched"].update({"replays": len(runs), "p99_ms_median": float(np.median(p99s)),
                           "p99_ms_range": [p99s[0], p99s[-1]],
                           "p50_ms_range": [min(r["p50_ms"] for r in runs), max(r["p50_ms"] for r in runs)],
                           "value_range": [min(r["value"] for r in runs), max(r["value"] for r in runs)],
                           "launches": int(st.launches), "gpu_busy_s": st.gpu_ms / 1e3})
    with Server(max_active=policies["one_per_launch"], chunk_steps=50, hbm_budget_bytes=SERVE_BUDGET) as srv:
        out["one_per_launch"] = run_trace(srv, pool, trace, SERVE_WARMUP, cap_s=20.0)
        st = srv.stats()
        out["one_per_launch"]["launches"] = int(st.launches)
    b, o = out["batched"], out["one_per_launch"]
    if b.get("value") and o.get("value"):
        out["batched_over_one_per_launch"] = b["value"] / o["value"]
    # capacity sweep: shorter traces of the same recipe at higher / lower rates
    cap = {"p99_bound_ms": SERVE_P99_BOUND_MS, "rule": "completed work >= 95 % of offered and p99 <= bound",
           "requests_per_rate": f"{SERVE_SWEEP_SECONDS:g} s of arrivals, 200 .. 1,600 requests, first 10 % warm-up"}
    main = {"batched": b, "one_per_launch": o}
    for name, rates in SERVE_SWEEP.items():
        sweep = {f"{SERVE_LAMBDA:g}": {k: main[name].get(k) for k in ("value", "offered", "p50_ms", "p99_ms")} |
                 {"keeps_up": keeps_up(main[name])}}
        for lam in rates:                    # a fresh server per rate: no backlog carries over
            n_req = sweep_requests(lam)
            tr = serve_trace(n_req, seed=11, lam=lam, pool=1600)
            with Server(max_active=policies[name], chunk_steps=50, hbm_budget_bytes=SERVE_BUDGET) as srv:
                r = run_trace(srv, pool, tr, n_req // 10, cap_s=25.0)
            ok = bool(r.get("completed")) and keeps_up(r)
            sweep[f"{lam:g}"] = {k: r.get(k) for k in ("value", "offered", "p50_ms", "p99_ms", "completed",
                                                       "measured_of")} | {"keeps_up": ok}
        ok_rates = sorted(float(k) for k, v in sweep.items() if v["keeps_up"])
        # capacity: the highest rate below which every swept rate keeps up
        best = None
        for lam in sorted(float(k) for k in sweep):
            if not sweep[f"{lam:g}"]["keeps_up"]:
                break
            best = lam
        cap[name] = {"req_per_s": best, "ceiling": max(v["value"] or 0.0 for v in sweep.values()),
                     "rates_kept_up": ok_rates, "sweep": sweep}
    out["capacity"] = cap
    return out


# ------------------------------------------------- CPU oracle (baseline) ----
def oracle_rate(n_envs: int, n_steps: int, threads: int, seed: int = 1) -> tuple[float, float]:
    """Times the FP64 oracle on the first n_envs envs of the workload for
    n_steps steps; returns (vehicle-steps/s, seconds)."""
    import oracle as O
    from paper_2305_16510_gb300 import workloads as W
    w = W.scaled(W.WORKLOADS[WORKLOAD], n_envs)
    inp = W.make_inputs(w, seed)
    world = O.World(n_envs=n_envs, substeps_per_step=w.substeps_per_step, integrator=w.integrator,
                    n_obs=w.n_obstacles, dt=w.dt, motor_tau=w.motor_tau, drag=w.drag)
    fl = O.make_fleet(world, body=inp.body.astype(np.float64), modes=inp.modes,
                      targets=inp.targets.astype(np.float64), boxes=inp.boxes.astype(np.float64), seed=seed)
    O.reset(world, fl, None, seed)
    t0 = time.perf_counter()
    O.rollout(world, fl, n_steps, n_threads=threads)
    dt = time.perf_counter() - t0
    return n_envs * n_steps / dt, dt


def _oracle_fleet(w, seed: int):
    """Oracle world and fleet of a workload, reset with its Philox draw."""
    import oracle as O
    from paper_2305_16510_gb300 import workloads as W
    inp = W.make_inputs(w, seed)
    world = O.World(n_envs=w.n_envs, substeps_per_step=w.substeps_per_step, integrator=w.integrator,
                    n_obs=w.n_obstacles, n_quad=w.n_quad, n_hexa=w.n_hexa, n_octo=w.n_octo, dt=w.dt,
                    motor_tau=w.motor_tau, drag=w.drag)
    fl = O.make_fleet(world, body=inp.body.astype(np.float64), modes=inp.modes,
                      targets=inp.targets.astype(np.float64),
                      boxes=None if inp.boxes is None else inp.boxes.astype(np.float64), seed=seed)
    O.reset(world, fl, None, seed)
    return world, fl, inp


def cpu_baseline_rows(parts, target_s: float = 3.0) -> dict:
    """The oracle, as it stands, on bounded samples of the other measured
    workloads (about target_s seconds each), in those lines' units."""
    import math
    import oracle as O
    from paper_2305_16510_gb300 import workloads as W
    threads = os.cpu_count() or 1
    rows = {}
    if "mixed" in parts:           # quad / hexa / octo, drag, randomised bodies, SIE (no reset masks)
        w = W.scaled(W.WORKLOADS["mixed"], 8192)
        world, fl, _ = _oracle_fleet(w, 1)
        t0 = time.perf_counter()
        O.rollout(world, fl, 10, n_threads=threads)
        k = max(10, int(10 * target_s / (time.perf_counter() - t0)))
        t0 = time.perf_counter()
        O.rollout(world, fl, k, n_threads=threads)
        dt = time.perf_counter() - t0
        rows["mixed"] = {"value": w.n_envs * k / dt, "unit": UNIT, "cores": threads,
                         "sample": f"{w.n_envs} envs x {k} steps ({dt:.1f} s, FP64)"}
    if "depth" in parts:           # 270 x 480, 87 deg, 10 m, 16 boxes per environment
        w = W.scaled(W.WORKLOADS[WORKLOAD], 64)
        world, fl, _ = _oracle_fleet(w, 1)
        t0 = time.perf_counter()
        O.render_depth(fl.state, fl.boxes, [0], 480, 270, math.radians(87), 10.0)
        k = max(1, min(64, int(target_s / (time.perf_counter() - t0))))
        t0 = time.perf_counter()
        O.render_depth(fl.state, fl.boxes, list(range(k)), 480, 270, math.radians(87), 10.0)
        dt = time.perf_counter() - t0
        rows["depth"] = {"value": k / dt, "unit": "depth frames/s", "cores": 1,
                         "sample": f"{k} cameras x 270 x 480, 16 boxes ({dt:.1f} s, FP64, 1 thread)"}
    if "task" in parts:            # reach task: commands, one SIE step, score, re-draw, observe
        n = 8192
        w = W.Workload("reach", n, 1, 0, 0, n, 0, 0, mode_mix=(W.MODE_ATT_THRUST,))
        world, fl, _ = _oracle_fleet(w, 1)
        rng = np.random.default_rng(1)
        goals = rng.uniform(-1.0, 1.0, (3, n))
        from paper_2305_16510_gb300 import _abi
        cfg = _abi.ag_reach_config_default()
        scale, offset = np.array(cfg.action_scale[:]), np.array(cfg.action_offset[:])
        steps = np.zeros(n, np.uint32)

        def task_step():
            nonlocal steps
            act = rng.uniform(-1.0, 1.0, (4, n))
            fl.targets[:] = offset[:, None] + scale[:, None] * np.clip(act, -1.0, 1.0)
            col, _ = O.rollout(world, fl, 1, n_threads=threads)
            _, _, done = O.reach_task(fl.state, goals, col, steps + 1)
            O.reset(world, fl, (done == 1) & (col == 0), 1)
            O.reach_task(fl.state, goals, col, steps + 1)
            steps = np.where(done == 1, 0, steps + 1).astype(np.uint32)

        t0 = time.perf_counter()
        task_step()
        k = max(2, int(target_s / (time.perf_counter() - t0)))
        t0 = time.perf_counter()
        for _ in range(k):
            task_step()
        dt = time.perf_counter() - t0
        rows["task"] = {"value": n * k / dt, "unit": "task env-steps/s", "cores": threads,
                        "sample": f"{n} envs x {k} task steps ({dt:.1f} s, FP64, rollout on {threads} threads)"}
    if "adjoint" in parts:         # the oracle's gradient: forward-mode passes, one per direction
        w = W.WORKLOADS["adjoint"]
        n, H = 512, w.horizon
        wv = W.scaled(w, n)
        world, fl, inp = _oracle_fleet(wv, 1)
        gains = world.gains12()
        goal = inp.targets[0:3].astype(np.float64)
        eye13, eye12 = np.eye(13), np.eye(12)

        def gradient(i):
            args = (world, 4, int(fl.modes[i]), fl.targets[:, i], fl.body[:, i], fl.state[:, i], fl.motors[:4, i])
            for d in range(13):
                O.vehicle_loss_jvp(*args, gains, eye13[d], np.zeros(12), H, goal[:, i])
            for d in range(12):
                O.vehicle_loss_jvp(*args, gains, np.zeros(13), eye12[d], H, goal[:, i])

        t0 = time.perf_counter()
        gradient(0)
        k = max(1, min(n, int(target_s / (time.perf_counter() - t0))))
        t0 = time.perf_counter()
        for i in range(k):
            gradient(i)
        dt = time.perf_counter() - t0
        rows["adjoint"] = {"value": k * H / dt, "unit": "vehicle-steps/s (forward + gradient)", "cores": 1,
                           "sample": f"{k} vehicles x {H} steps, 25 forward-mode passes each (13 state + 12 gain "
                                     f"directions; the oracle has no reverse mode) ({dt:.1f} s, FP64, 1 thread)"}
    return rows


def cpu_baseline(target_s: float = 12.0) -> dict:
    threads = os.cpu_count() or 1
    n_envs = 8192
    rate, _ = oracle_rate(n_envs, 20, threads)
    n_steps = max(2, int(target_s * rate / n_envs))
    rate, secs = oracle_rate(n_envs, n_steps, threads)
    # one host thread, on a sample of about 3 s
    n1 = 512
    r1, _ = oracle_rate(n1, 5, 1)
    steps1 = max(2, int(3.0 * r1 / n1))
    r1, s1 = oracle_rate(n1, steps1, 1)
    return {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n_envs} envs x {n_steps} steps of the same workload ({secs:.1f} s, FP64, {threads} threads)",
            "single_thread": {"value": r1, "unit": UNIT,
                              "sample": f"{n1} envs x {steps1} steps ({s1:.1f} s, FP64, 1 thread)"}}


def reference_arm(args) -> dict | None:
    world, rank, _ = dist_env()
    if rank != 0:
        return None
    threads = os.cpu_count() or 1
    n_envs = 4096
    rate0, _ = oracle_rate(n_envs, 50, threads)
    n_steps = max(1, int(4.0 * rate0 / n_envs))       # ~4 s of oracle work per bench step
    for _ in range(args.warmup):
        oracle_rate(n_envs, 1, threads)
    total_units, total_s = 0, 0.0
    for _ in range(args.steps):
        r, s = oracle_rate(n_envs, n_steps, threads, seed=1)
        total_units += n_envs * n_steps
        total_s += s
    value = total_units / total_s
    sample = f"{n_envs} envs x {n_steps} steps per bench step (FP64 oracle, {threads} threads)"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT, "n_envs": 1 << 20, "steps_per_call": STEPS_PER_CALL,
                       "parallelism": "host threads"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


PARTS = ("fused", "plain", "e2e", "paper", "mixed", "depth", "task", "adjoint", "serve")


def make_parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--envs", type=int, default=0, help="reduced fleet size (default: the full workload)")
    ap.add_argument("--steps-per-call", type=int, default=STEPS_PER_CALL)
    ap.add_argument("--parts", default=",".join(PARTS))
    ap.add_argument("--seed", type=int, default=1, help="input seed of rank 0 (rank r uses seed + r)")
    return ap


DETAIL_DIR = os.path.join(ROOT, "gpurun_out")


def detail_path(parts: str) -> str:
    """Side file of a run: bench_detail.json for every part, else named by the parts."""
    if set(parts.split(",")) == set(PARTS):
        return os.path.join(DETAIL_DIR, "bench_detail.json")
    return os.path.join(DETAIL_DIR, "bench_detail_" + "_".join(sorted(parts.split(","))) + ".json")


def _sig(x, digits: int = 4):
    """x rounded to `digits` significant digits (recursively in lists and dicts)."""
    if isinstance(x, bool) or x is None or isinstance(x, (int, str)):
        return x
    if isinstance(x, float):
        return float(f"{x:.{digits}g}")
    if isinstance(x, (list, tuple)):
        return [_sig(v, digits) for v in x]
    if isinstance(x, dict):
        return {k: _sig(v, digits) for k, v in x.items()}
    return x


def _pick(d: dict | None, *keys):
    if not d:
        return None
    return {k: d[k] for k in keys if k in d}


def compact_line(res: dict) -> dict:
    """The printed JSON line: the contract's keys plus the headline figures of
    every part, each number to 4 significant digits, short enough (about
    1.4 KB) to be kept whole by a reader of the output's tail. Everything
    else (workload texts, latency histograms, the sweep, per-row CPU
    baselines) goes to the side file."""
    r = res
    out = {k: r[k] for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                             "higher_is_better", "scaling", "vs_baseline", "dtype") if k in r}
    out["data"] = "synthetic"
    cfg = r["config"]
    nq = cfg["n_envs"]
    out["config"] = {"workload": (f"{nq >> 20 if nq % (1 << 20) == 0 else nq}{'M' if nq % (1 << 20) == 0 else ''} "
                                  f"quads,3 modes,RK4x{cfg['substeps_per_step']},"
                                  f"{cfg['boxes_per_env']} OBB,{cfg['steps_per_call']} steps/call"),
                     "l2": "inputs>L2"}
    rf = r["roofline"]
    out["roofline"] = {**_pick(rf, "bound", "achieved", "peak", "unit", "frac", "traffic"),
                       "frac_performed": rf["frac_performed"],
                       "fma_chain_tflops": rf["fma_chain_check"]["packed_tflops"]}
    if "cpu_baseline" in r:
        cb = r["cpu_baseline"]
        out["cpu_baseline"] = {**_pick(cb, "value", "unit", "cores", "kind"), "sample": cb["sample"].split(" of ")[0]}
    out["clocks"] = _pick(r["clocks"], "sm_mhz", "sm_max_mhz", "reasons")
    if "e2e" in r:
        out["e2e"] = r["e2e"]
    out["gpu_launches"] = r["gpu_launches"]
    out["range"] = r["range"]
    if "plain" in r:
        out["plain"] = _pick(r["plain"], "value", "fused_over_plain")
    if "serving" in r:
        sv = r["serving"]
        b, o = sv.get("batched", {}), sv.get("one_per_launch", {})
        cap = sv.get("capacity", {})
        out["serving"] = {"batched": {**_pick(b, "value", "p50_ms"), "p99_ms": b.get("p99_ms_median"),
                                      "p99_range": b.get("p99_ms_range")},
                          "one_per_launch": _pick(o, "value", "p50_ms", "p99_ms"),
                          "capacity": {"p99_bound_ms": cap.get("p99_bound_ms"),
                                       "batched": (cap.get("batched") or {}).get("req_per_s"),
                                       "one_per_launch": (cap.get("one_per_launch") or {}).get("req_per_s"),
                                       "ceiling": [(cap.get(k) or {}).get("ceiling")
                                                   for k in ("batched", "one_per_launch")]}}
    for key in ("mixed", "paper_shape"):
        if key in r:
            out[key] = _pick(r[key], "value", "alu_frac", "range")
    if "depth" in r:
        out["depth"] = _pick(r["depth"], "value", "alu_frac")
    if "task" in r:
        out["task"] = _pick(r["task"], "value", "hbm_frac")
    if "adjoint" in r:
        a = r["adjoint"]
        out["adjoint"] = {"value": a["value"], "alu_fwd": a["alu_frac_record"], "alu_bwd": a["alu_frac_backward"],
                          "range": a["range"]}
    head = {k: out[k] for k in list(out)[:list(out).index("range") + 1]}
    parts = {k: out[k] for k in list(out)[list(out).index("range") + 1:]}
    return {**_sig(head, 4), **_sig(parts, 3)}


def dumps_compact(x) -> str:
    """JSON with no spaces and floats in %.4g form (exponents without '+' or
    leading zeros, e.g. 1.373e10): valid JSON, about a third shorter."""
    if isinstance(x, dict):
        return "{" + ",".join(json.dumps(str(k)) + ":" + dumps_compact(v) for k, v in x.items()) + "}"
    if isinstance(x, (list, tuple)):
        return "[" + ",".join(dumps_compact(v) for v in x) + "]"
    if isinstance(x, float) and np.isfinite(x):
        t = f"{x:.4g}"
        if "e" in t:
            m, e = t.split("e")
            t = f"{m}e{int(e)}"
        return t
    if isinstance(x, float):
        return "null"
    return json.dumps(x)


def write_detail(res: dict, path: str) -> None:
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(res, f, indent=1)
    except OSError as e:
        print(f"bench: could not write {path}: {e}", file=sys.stderr)


def main():
    ap = make_parser()
    args = ap.parse_args()
    unknown = set(args.parts.split(",")) - set(PARTS)
    if unknown:
        ap.error(f"unknown --parts: {sorted(unknown)} (choose from {', '.join(PARTS)})")
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        out = reference_arm(args)
        if out is not None:
            print(dumps_compact(out), flush=True)
        return
    out = gpu_arm(args)
    if out is None:
        return
    world, _, _ = dist_env()
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline()
        out["cpu_baseline"]["rows"] = cpu_baseline_rows(set(args.parts.split(",")))
    write_detail(out, detail_path(args.parts))
    print(dumps_compact(compact_line(out)), flush=True)


if __name__ == "__main__":
    main()
