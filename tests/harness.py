"""Shared test helpers: run the CUDA path and the oracle on the same inputs.

Inputs come from paper_2305_16510_gb300.workloads (seeded numpy draws); the
initial states come from each side's own Philox reset. Nothing here computes
a simulation step itself except `box_margin`, a plain numpy distance used only
to flag collision near-ties where float32 and float64 may legitimately
disagree.
"""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2305_16510_gb300 import workloads as W

G = 9.81


def oracle_world(w: W.Workload) -> O.World:
    return O.World(n_envs=w.n_envs, substeps_per_step=w.substeps_per_step, integrator=w.integrator,
                   n_obs=w.n_obstacles, n_quad=w.n_quad, n_hexa=w.n_hexa, n_octo=w.n_octo, dt=w.dt,
                   motor_tau=w.motor_tau, drag=w.drag)


def gpu_fleet(w: W.Workload, inp: W.Inputs, seed: int):
    from paper_2305_16510_gb300.fleet import Fleet
    fl = Fleet(w.n_envs, substeps_per_step=w.substeps_per_step, integrator=w.integrator, n_obstacles=w.n_obstacles,
               n_hexa=w.n_hexa, n_octo=w.n_octo, dt=w.dt, motor_tau=w.motor_tau, drag=w.drag, seed=seed)
    fl.set_body(inp.body)
    fl.set_commands(inp.modes, inp.targets)
    if inp.boxes is not None:
        fl.set_obstacles(inp.boxes)
    return fl


def oracle_fleet_from(w: W.Workload, inp: W.Inputs, state, motors, epoch, seed: int) -> O.Fleet:
    """Oracle fleet at a given float32 state (widened exactly to float64)."""
    return O.make_fleet(oracle_world(w), state=np.asarray(state, dtype=np.float64),
                        motors=np.asarray(motors, dtype=np.float64), body=inp.body.astype(np.float64),
                        modes=inp.modes, targets=inp.targets.astype(np.float64), epoch=np.asarray(epoch),
                        boxes=None if inp.boxes is None else inp.boxes.astype(np.float64), seed=seed)


def subset(w: W.Workload, inp: W.Inputs, idx: np.ndarray):
    """Workload and inputs restricted to the sorted env indices idx (rotor
    types stay in contiguous quad / hexa / octo ranges)."""
    idx = np.asarray(idx)
    assert np.all(np.diff(idx) > 0)
    n_quad = int(np.sum(idx < w.n_quad))
    n_hexa = int(np.sum((idx >= w.n_quad) & (idx < w.n_quad + w.n_hexa)))
    w2 = W.Workload(**{**w.__dict__, "n_envs": len(idx), "n_quad": n_quad, "n_hexa": n_hexa,
                       "n_octo": len(idx) - n_quad - n_hexa})
    inp2 = W.Inputs(inp.modes[idx], inp.targets[:, idx], inp.body[:, idx],
                    None if inp.boxes is None else np.ascontiguousarray(inp.boxes[:, :, idx]))
    return w2, inp2


def attitude_error(q_a: np.ndarray, q_b: np.ndarray) -> np.ndarray:
    """Rotation angle between unit quaternions given as [4, n] arrays (w, x, y, z)."""
    qa = q_a / np.linalg.norm(q_a, axis=0)
    qb = q_b / np.linalg.norm(q_b, axis=0)
    d = np.abs(np.sum(qa * qb, axis=0))
    v = np.sqrt(np.maximum(0.0, 1.0 - np.minimum(d, 1.0) ** 2))
    return 2.0 * np.arctan2(v, d)


def box_margin(p: np.ndarray, boxes: np.ndarray, r: float = 0.2) -> np.ndarray:
    """min over boxes of (squared distance from p to the box) - r^2, per env.

    p: [3, n] float64, boxes: [n_obs, 10, n]. Used only to flag near-ties.
    """
    out = np.full(p.shape[1], np.inf)
    for k in range(boxes.shape[0]):
        c, h, q = boxes[k, 0:3], boxes[k, 3:6], boxes[k, 6:10]
        w, u = q[0], q[1:4]
        v = p - c
        t = 2.0 * np.cross(u, v, axis=0)
        d = v - w * t + np.cross(u, t, axis=0)
        e = d - np.clip(d, -h, h)
        out = np.minimum(out, np.sum(e * e, axis=0) - r * r)
    return out


def max_state_errors(gpu: np.ndarray, orc: np.ndarray):
    dp = np.max(np.abs(gpu[0:3].astype(np.float64) - orc[0:3]), axis=0)
    dv = np.max(np.abs(gpu[3:6].astype(np.float64) - orc[3:6]), axis=0)
    dang = attitude_error(gpu[6:10].astype(np.float64), orc[6:10])
    dw = np.max(np.abs(gpu[10:13].astype(np.float64) - orc[10:13]), axis=0)
    return dp, dv, dang, dw
