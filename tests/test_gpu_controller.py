"""The controller stage alone (ag_eval_controller) against the FP64 oracle.

Sec. IV: in each command mode the controller turns a state and a target
into the commanded collective thrust and moments (position tracking, body
velocity Eqs. 6-9, attitude and thrust Eqs. 1-5, or a direct wrench). The
states here cover every attitude (uniform on SO(3), upside down included),
fast body rates and velocities, a few exact hover states (f = m g, M = 0)
and states whose body x axis is vertical (the current yaw is then read from
R_10 = 0 and R_00 ~ 0, the same branch in float32 and float64).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2305_16510_gb300 import _abi
from paper_2305_16510_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GAINS = np.array([2, 2, 3, 2, 2, 2, 1.2, 1.2, 0.6, 0.2, 0.2, 0.1], dtype=np.float64)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2305_16510_gb300 import build
    build.build()


def _states(n, rng):
    st = np.zeros((13, n), np.float32)
    st[0:3] = rng.uniform(-3, 3, (3, n))
    st[3:6] = rng.normal(0.0, 1.5, (3, n))
    u1, u2, u3 = rng.uniform(size=(3, n))
    a, b = np.sqrt(1 - u1), np.sqrt(u1)
    st[6:10] = np.stack([b * np.cos(2 * np.pi * u3), a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2),
                         b * np.sin(2 * np.pi * u3)])
    st[10:13] = rng.normal(0.0, 2.0, (3, n))
    return st


def test_controller_matches_oracle_in_every_mode():
    n = 4096
    rng = np.random.default_rng(11)
    modes = (np.arange(n) % 4).astype(np.uint8)
    body = W.body(W.Workload("c", n, 1, 0, 0, n, 0, 0, mass_rand=0.2), rng)
    targets = W.targets(modes, rng, body[0].astype(np.float64))
    wrench_rows = modes == W.MODE_WRENCH
    targets[:, wrench_rows] = rng.normal(0.0, 1.0, (4, int(wrench_rows.sum()))).astype(np.float32)
    st = _states(n, rng)
    # exact hover in position mode: p = p_d, v = 0, yaw = psi_d, Omega = 0
    hover = np.flatnonzero(modes == W.MODE_POSITION)[:32]
    st[0:3, hover] = targets[0:3, hover]
    st[3:6, hover] = 0.0
    st[10:13, hover] = 0.0
    half = targets[3, hover].astype(np.float64) / 2
    st[6:10, hover] = np.stack([np.cos(half), 0 * half, 0 * half, np.sin(half)]).astype(np.float32)
    # body x axis vertical (pitch -90 deg), velocity and attitude modes
    vert = np.flatnonzero((modes == W.MODE_BODY_VEL) | (modes == W.MODE_ATT_THRUST))[:32]
    st[6:10, vert] = np.array([[1.0], [0.0], [1.0], [0.0]], np.float32)   # not unit: the controller normalises q

    from paper_2305_16510_gb300.fleet import Fleet
    fl = Fleet(n)
    fl.set_body(body)
    fl.set_commands(modes, targets)
    out = torch.empty((4, n), device=fl.device)
    _abi.ag_eval_controller(fl.ctx, torch.from_numpy(st).cuda(), out)
    got = out.cpu().numpy().astype(np.float64)
    # state NULL: the context's current state (set to the same states)
    fl.set_state(st)
    out2 = torch.empty((4, n), device=fl.device)
    _abi.ag_eval_controller(fl.ctx, None, out2)
    np.testing.assert_array_equal(out2.cpu().numpy(), got.astype(np.float32))
    np.testing.assert_array_equal(fl.eval_controller().cpu().numpy(), got.astype(np.float32))
    fl.close()

    ref = np.zeros((4, n))
    for i in range(n):
        ref[:, i] = O.controller(int(modes[i]), st[:, i].astype(np.float64), targets[:, i].astype(np.float64),
                                 body[:, i].astype(np.float64), GAINS)["fM"]
    err = np.abs(got - ref)
    tol = 1e-4 * (1.0 + np.abs(ref))
    bad = np.argwhere(err > tol)
    assert bad.size == 0, [(int(modes[j]), int(k), got[k, j], ref[k, j]) for k, j in bad[:8]]
    # hover: thrust m g and no moment
    np.testing.assert_allclose(got[0, hover], body[0, hover].astype(np.float64) * 9.81, rtol=1e-5)
    np.testing.assert_allclose(got[1:4, hover], 0.0, atol=1e-5)
    # wrench mode passes the targets through
    np.testing.assert_array_equal(got[:, wrench_rows].astype(np.float32), targets[:, wrench_rows])


def test_eval_controller_rejects_null_output():
    from paper_2305_16510_gb300.fleet import Fleet
    fl = Fleet(64)
    with pytest.raises(_abi.AgError) as e:
        _abi.ag_eval_controller(fl.ctx, None, None)
    assert e.value.status == _abi.AG_ERR_INVALID
    fl.close()
