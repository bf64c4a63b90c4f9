"""Seeded synthetic inputs of the fleet workloads.

This module only draws input arrays (commands, obstacles, body parameters,
reset masks) with numpy's seeded generator; it holds none of the
simulation's arithmetic and is shared by the tests, the bench and the
oracle runs so that both sides see the same inputs. Initial vehicle states
are NOT drawn here: they come from the library's Philox reset (ag_reset),
which the oracle reproduces bit for bit.

Recipes (sizes and distributions of the fleet workloads):
  parity      1,024 quads, position mode, targets U[-3, 3]^3 m, yaw U[-pi, pi),
              semi-implicit Euler, dt 0.01 s, 1 substep, no obstacles
  obstacles   1,048,576 quads, mode uniform over {position, body velocity,
              attitude+thrust} per env, RK4 with 4 substeps, 16 boxes per env:
              centres U[-5, 5]^3 m, half-extents U[0.1, 1] m, orientation
              uniform on SO(3) (Shoemake), sphere radius 0.2 m
  mixed       4,194,304 vehicles, 40 % quad / 40 % hexa / 20 % octo in
              contiguous ranges, mass and inertia x U[0.8, 1.2], motor lag
              0.03 s, drag 0.1, body-velocity targets U[-2, 2]^3 m/s, yaw rate
              U[-1, 1], 1 % Bernoulli reset mask every 50 steps
  paper_shape 131,072 quads, attitude or body-velocity command, no obstacles,
              1 substep (the fleet size of the paper's throughput figure)
  adjoint     65,536 quads, position mode (targets as in parity), semi-implicit
              Euler, 1 substep, horizon 256 steps, goals = the position
              targets, checkpoint every 32 steps
Targets per mode: position U[-3, 3]^3 and yaw U[-pi, pi); body velocity
U[-2, 2]^3 and yaw rate U[-1, 1]; attitude roll and pitch U[-30, 30] deg,
yaw rate U[-1, 1], collective thrust U[0.5, 1.5] m g.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

MODE_POSITION, MODE_BODY_VEL, MODE_ATT_THRUST, MODE_WRENCH = 0, 1, 2, 3
NOMINAL_MASS = 0.75
NOMINAL_INERTIA = (0.007, 0.007, 0.012)
G = 9.81


@dataclass
class Workload:
    name: str
    n_envs: int
    substeps_per_step: int
    integrator: int            # 0 semi-implicit Euler, 1 RK4
    n_obstacles: int
    n_quad: int
    n_hexa: int
    n_octo: int
    motor_tau: float = 0.03
    drag: float = 0.0
    dt: float = 0.01
    horizon: int = 100         # steps the workload is defined over
    mass_rand: float = 0.0     # +- fraction
    mode_mix: tuple = (MODE_POSITION,)
    reset_every: int = 0       # steps between Bernoulli reset masks (0 = none)
    reset_prob: float = 0.0


WORKLOADS = {
    "parity": Workload("parity", 1024, 1, 0, 0, 1024, 0, 0, horizon=100),
    "obstacles": Workload("obstacles", 1 << 20, 4, 1, 16, 1 << 20, 0, 0, horizon=1000,
                          mode_mix=(MODE_POSITION, MODE_BODY_VEL, MODE_ATT_THRUST)),
    "mixed": Workload("mixed", 4194304, 1, 0, 0, 1677722, 1677722, 838860, drag=0.1, horizon=500, mass_rand=0.2,
                      mode_mix=(MODE_BODY_VEL,), reset_every=50, reset_prob=0.01),
    "paper_shape": Workload("paper_shape", 1 << 17, 1, 0, 0, 1 << 17, 0, 0, horizon=100,
                            mode_mix=(MODE_BODY_VEL, MODE_ATT_THRUST)),
    "adjoint": Workload("adjoint", 65536, 1, 0, 0, 65536, 0, 0, horizon=256, mode_mix=(MODE_POSITION,)),
}


def scaled(w: Workload, n_envs: int) -> Workload:
    """Same recipe at a different fleet size (type fractions kept)."""
    frac_h = w.n_hexa / w.n_envs
    frac_o = w.n_octo / w.n_envs
    n_hexa = int(round(n_envs * frac_h))
    n_octo = int(round(n_envs * frac_o))
    return Workload(**{**w.__dict__, "n_envs": n_envs, "n_quad": n_envs - n_hexa - n_octo, "n_hexa": n_hexa,
                       "n_octo": n_octo})


def modes(w: Workload, rng: np.random.Generator) -> np.ndarray:
    mix = np.asarray(w.mode_mix, dtype=np.uint8)
    return mix[rng.integers(0, len(mix), size=w.n_envs)].astype(np.uint8)


def targets(mode_arr: np.ndarray, rng: np.random.Generator, mass: np.ndarray | None = None) -> np.ndarray:
    """float32 [4, n] targets for each env's mode."""
    n = mode_arr.shape[0]
    m = np.full(n, NOMINAL_MASS) if mass is None else mass
    t = np.zeros((4, n), dtype=np.float64)
    pos = mode_arr == MODE_POSITION
    vel = mode_arr == MODE_BODY_VEL
    att = mode_arr == MODE_ATT_THRUST
    t[0:3, pos] = rng.uniform(-3, 3, size=(3, pos.sum()))
    t[3, pos] = rng.uniform(-np.pi, np.pi, size=pos.sum())
    t[0:3, vel] = rng.uniform(-2, 2, size=(3, vel.sum()))
    t[3, vel] = rng.uniform(-1, 1, size=vel.sum())
    a30 = np.radians(30.0)
    t[0:2, att] = rng.uniform(-a30, a30, size=(2, att.sum()))
    t[2, att] = rng.uniform(-1, 1, size=att.sum())
    t[3, att] = rng.uniform(0.5, 1.5, size=att.sum()) * m[att] * G
    return t.astype(np.float32)


def boxes(n_envs: int, n_obs: int, rng: np.random.Generator) -> np.ndarray:
    """float32 [n_obs, 10, n]: centre, half-extents, unit quaternion (w, x, y, z)."""
    out = np.zeros((n_obs, 10, n_envs), dtype=np.float32)
    for k in range(n_obs):
        out[k, 0:3] = rng.uniform(-5, 5, size=(3, n_envs))
        out[k, 3:6] = rng.uniform(0.1, 1.0, size=(3, n_envs))
        u1, u2, u3 = rng.uniform(size=(3, n_envs))
        a, b = np.sqrt(1 - u1), np.sqrt(u1)
        q = np.stack([b * np.cos(2 * np.pi * u3), a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2),
                      b * np.sin(2 * np.pi * u3)])
        out[k, 6:10] = q
    return out


def body(w: Workload, rng: np.random.Generator) -> np.ndarray:
    """float32 [4, n]: mass and diagonal inertia, scaled by U[1 - r, 1 + r]."""
    n = w.n_envs
    out = np.empty((4, n), dtype=np.float32)
    out[0] = NOMINAL_MASS
    out[1:4] = np.asarray(NOMINAL_INERTIA, dtype=np.float64)[:, None]
    if w.mass_rand > 0:
        out[0] *= rng.uniform(1 - w.mass_rand, 1 + w.mass_rand, size=n)
        out[1:4] *= rng.uniform(1 - w.mass_rand, 1 + w.mass_rand, size=(3, n))
    return out


def reset_mask(n_envs: int, p: float, rng: np.random.Generator) -> np.ndarray:
    return (rng.uniform(size=n_envs) < p).astype(np.uint8)


@dataclass
class Inputs:
    modes: np.ndarray
    targets: np.ndarray
    body: np.ndarray
    boxes: np.ndarray | None


def make_inputs(w: Workload, seed: int) -> Inputs:
    rng = np.random.default_rng(seed)
    b = body(w, rng)
    md = modes(w, rng)
    tg = targets(md, rng, b[0].astype(np.float64))
    bx = boxes(w.n_envs, w.n_obstacles, rng) if w.n_obstacles > 0 else None
    return Inputs(md, tg, b, bx)
