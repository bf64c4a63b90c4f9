"""Reach-a-setpoint task (ag_reach_step) vs the oracle, one step at a time.

Sec. I: policies fly the vehicle to a goal setpoint through the attitude or
the velocity command interface. Each task step maps actions to commands,
takes one fleet step, scores it, ends episodes (collision, distance, step
limit), re-draws the episodes that ended without a collision and observes
the new state. The oracle side composes the same definition from its own
rollout, reset and task functions, starting every step from the GPU's
float32 state (teacher forcing).
"""
import numpy as np
import pytest
import torch

import oracle as O
from harness import box_margin, oracle_fleet_from, oracle_world
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


def _cfg(mode, max_steps, max_dist):
    c = _abi.ag_reach_config_default()
    c.command_mode = mode
    if mode == _abi.AG_MODE_BODY_VEL:
        c.action_scale[:] = [2.0, 2.0, 2.0, 1.0]
        c.action_offset[:] = [0.0, 0.0, 0.0, 0.0]
    c.max_steps, c.max_dist = max_steps, max_dist
    return c


def _params(c):
    return dict(w_v=c.w_v, w_w=c.w_omega, crash=c.crash, max_dist=c.max_dist, max_steps=c.max_steps)


CASES = [
    # RK4, 4 substeps, boxes (collisions end episodes), attitude interface
    (W.Workload("reach_att", 3000, 4, 1, 8, 3000, 0, 0), _abi.AG_MODE_ATT_THRUST, False),
    # the same with obstacle re-placement on every reset, quad / hexa / octo
    (W.Workload("reach_redraw", 3000, 4, 1, 8, 1200, 1200, 600), _abi.AG_MODE_ATT_THRUST, True),
    # semi-implicit Euler, quad / hexa / octo, no boxes, velocity interface
    (W.Workload("reach_vel", 2500, 1, 0, 0, 1000, 1000, 500, drag=0.1), _abi.AG_MODE_BODY_VEL, False),
    # an odd fleet size (1001 = 7 x 128 + 105: a ragged last block), quad / hexa
    (W.Workload("reach_vel_odd", 1001, 1, 0, 0, 501, 500, 0), _abi.AG_MODE_BODY_VEL, False),
    # quad / hexa without boxes, full blocks only (2048 = 16 x 128), RK4 x 2, attitude interface
    (W.Workload("reach_att_hexa", 2048, 2, 1, 0, 1024, 1024, 0), _abi.AG_MODE_ATT_THRUST, False),
]
ENV_MIN, ENV_MAX = (-5.0, -5.0, -5.0), (5.0, 5.0, 5.0)


def _box_specs(n_obs):
    kw = [dict(pos_min=(0.2, 0.2, 0.2), pos_max=(0.8, 0.8, 0.8), euler_min=(-1, -1, -3), euler_max=(1, 1, 3),
               lock=0, fixed=[0.0] * 6) for _ in range(n_obs)]
    return [_abi.box_randomization(**k) for k in kw], [O.box_rand(**k) for k in kw]


@pytest.mark.parametrize("w,mode,redraw", CASES, ids=[c[0].name for c in CASES])
def test_reach_step_matches_oracle(w, mode, redraw):
    from harness import gpu_fleet
    seed = 23
    inp = W.make_inputs(w, seed)
    fl = gpu_fleet(w, inp, seed)
    world = oracle_world(w)
    if redraw:
        sg, so = _box_specs(w.n_obstacles)
        fl.set_obstacle_randomization(ENV_MIN, ENV_MAX, sg)
        world = O.World(**{**world.__dict__, "env_min": ENV_MIN, "env_max": ENV_MAX, "box_specs": so})
    world_free = O.World(**{**world.__dict__, "n_obs": 0, "box_specs": None})
    rng = np.random.default_rng(5)
    goals = rng.uniform(-1.0, 1.0, (3, w.n_envs)).astype(np.float32)
    cfg = _cfg(mode, max_steps=3, max_dist=3.0)
    fl.reset(None, seed)
    _abi.ag_reach_begin(fl.ctx, cfg, torch.from_numpy(goals).cuda())
    dev = fl.device
    obs = torch.empty((w.n_envs, 13), device=dev)
    rew = torch.empty((w.n_envs,), device=dev)
    done = torch.empty((w.n_envs,), dtype=torch.uint8, device=dev)
    modes = np.full(w.n_envs, mode, np.uint8)
    scale, offset = np.array(cfg.action_scale[:]), np.array(cfg.action_offset[:])
    steps = np.zeros(w.n_envs, np.uint32)
    seen = {"collided": 0, "far": 0, "timeout": 0}
    for _ in range(7):
        s0, m0, e0 = _np(fl.state()), _np(fl.motors()), _np(fl.epoch()).astype(np.uint32)
        b0 = _np(fl.obstacles()) if w.n_obstacles else None
        act = rng.uniform(-1.3, 1.3, (w.n_envs, 4)).astype(np.float32)
        _abi.ag_reach_step(fl.ctx, torch.from_numpy(act).to(dev), obs, rew, done)
        g_obs, g_rew, g_done = _np(obs), _np(rew), _np(done)
        g_col = _np(fl.events()[0])
        g_epoch = _np(fl.epoch())
        # oracle: commands, one step, score, end, re-draw, observe
        tgt = (offset[:, None] + scale[:, None] * np.clip(act.T.astype(np.float64), -1.0, 1.0))
        cur = W.Inputs(modes, tgt, inp.body, b0)
        orc = oracle_fleet_from(w, cur, s0, m0, e0, seed)
        ocol, _ = O.rollout(world, orc, 1)
        nxt = steps + 1
        _, o_rew, o_done = O.reach_task(orc.state, goals, ocol, nxt, **_params(cfg))
        dist = np.linalg.norm(orc.state[0:3] - goals, axis=0)
        O.reset(world, orc, (o_done == 1) & (ocol == 0), seed)
        o_obs = O.reach_task(orc.state, goals, ocol, nxt, **_params(cfg))[0].T
        # float32 / float64 near-ties of the two decisions are left out
        ok = np.abs(dist - cfg.max_dist) >= 1e-4
        if w.n_obstacles:
            pre = oracle_fleet_from(w, W.Inputs(modes, tgt, inp.body, None), s0, m0, e0, seed)
            O.rollout(world_free, pre, 1)
            ok &= np.abs(box_margin(pre.state[0:3], b0.astype(np.float64))) >= 1e-5
        assert ok.mean() > 0.99
        np.testing.assert_array_equal(g_col[ok], ocol[ok])
        np.testing.assert_array_equal(g_done[ok], o_done[ok])
        np.testing.assert_array_equal(g_epoch[ok], orc.epoch[ok])
        if w.n_obstacles:   # re-drawn (or kept) boxes, bit for bit
            np.testing.assert_array_equal(_np(fl.obstacles())[:, :, ok], orc.boxes[:, :, ok].astype(np.float32))
        hit = ok & (ocol == 1)
        assert np.all(g_rew[hit] == np.float32(-cfg.crash))
        free = ok & (ocol == 0)
        np.testing.assert_allclose(g_rew[free], o_rew[free], rtol=1e-4, atol=1e-4)
        # observations; q and -q describe one attitude, so near w = 0 the sign may differ
        d = np.abs(g_obs[ok].astype(np.float64) - o_obs[ok])
        tol = 1e-4 * (1.0 + np.abs(o_obs[ok]))
        flip = np.abs(o_obs[ok, 6]) < 1e-4
        d[flip, 6:10] = np.abs(np.abs(g_obs[ok][flip, 6:10]) - np.abs(o_obs[ok][flip, 6:10]))
        assert np.all(d <= tol), float((d - tol).max())
        # episodes that ended restart from the reset draw: their observation is exact up to the goal subtraction
        ended = ok & (o_done == 1)
        np.testing.assert_allclose(g_obs[ended], o_obs[ended], atol=2e-6)
        seen["collided"] += int(hit.sum())
        seen["far"] += int((free & (dist > cfg.max_dist)).sum())
        seen["timeout"] += int((free & (nxt >= cfg.max_steps) & (dist <= cfg.max_dist)).sum())
        steps = np.where(g_done == 1, 0, steps + 1).astype(np.uint32)
    assert seen["far"] > 0 and seen["timeout"] > 0
    if w.n_obstacles:
        assert seen["collided"] > 0
    fl.close()


def test_reach_env_reset_and_autoreset():
    from paper_2305_16510_gb300.task import ReachEnv
    n = 4096
    env = ReachEnv(n, seed=9)
    obs = env.reset()
    st = _np(env.fleet.state())
    o_obs = O.reach_task(st.astype(np.float64), np.zeros((3, n)), np.zeros(n, np.uint8), np.zeros(n, np.uint32))[0].T
    np.testing.assert_allclose(_np(obs), o_obs, atol=1e-7)
    assert np.all(_np(obs)[:, 6] >= 0.0)
    ep0 = _np(env.fleet.epoch()).copy()
    ended = np.zeros(n, np.int64)
    hover = torch.zeros((n, 4), device=env.device)   # level attitude, hover thrust
    for t in range(env.task.max_steps):
        obs, rew, done, info = env.step(hover)
        ended += _np(done)
        assert torch.isfinite(rew).all()
    # every episode hit the step limit at the latest, and restarted with a new draw
    assert np.all(ended >= 1)
    assert np.all(_np(env.fleet.epoch()) - ep0 == ended)
    env.close()


def test_reach_errors():
    from paper_2305_16510_gb300.fleet import Fleet
    fl = Fleet(256)
    buf = torch.zeros((256 * 13 + 8,), device=fl.device)
    with pytest.raises(_abi.AgError) as e:
        _abi.ag_reach_step(fl.ctx, buf, buf, buf, buf)
    assert e.value.status == _abi.AG_ERR_STATE
    bad = _abi.ag_reach_config_default()
    bad.command_mode = _abi.AG_MODE_POSITION
    with pytest.raises(_abi.AgError) as e:
        _abi.ag_reach_begin(fl.ctx, bad, torch.zeros((3, 256), device=fl.device))
    assert e.value.status == _abi.AG_ERR_INVALID
    _abi.ag_reach_begin(fl.ctx, _abi.ag_reach_config_default(), torch.zeros((3, 256), device=fl.device))
    with pytest.raises(_abi.AgError) as e:   # rejected on the host before any launch
        _abi.ag_reach_step(fl.ctx, buf.data_ptr() + 4, buf, buf, buf)
    assert e.value.status == _abi.AG_ERR_INVALID
    fl.close()


@pytest.mark.parametrize("n", [1, 3, 33])
def test_reach_step_on_tiny_and_ragged_fleets(n):
    """Fleets smaller than a warp or one lane past it: one task step against
    the oracle's composition (the observation rows of a partly empty warp)."""
    from harness import gpu_fleet
    seed = 8
    w = W.Workload("reach_small", n, 1, 0, 0, n, 0, 0)
    inp = W.make_inputs(w, seed)
    fl = gpu_fleet(w, inp, seed)
    world = oracle_world(w)
    rng = np.random.default_rng(n)
    goals = rng.uniform(-1.0, 1.0, (3, n)).astype(np.float32)
    cfg = _cfg(_abi.AG_MODE_ATT_THRUST, max_steps=1, max_dist=3.0)
    fl.reset(None, seed)
    _abi.ag_reach_begin(fl.ctx, cfg, torch.from_numpy(goals).cuda())
    dev = fl.device
    obs = torch.full((n, 13), np.nan, device=dev)
    rew = torch.empty((n,), device=dev)
    done = torch.empty((n,), dtype=torch.uint8, device=dev)
    s0, m0, e0 = _np(fl.state()), _np(fl.motors()), _np(fl.epoch()).astype(np.uint32)
    act = rng.uniform(-1.0, 1.0, (n, 4)).astype(np.float32)
    _abi.ag_reach_step(fl.ctx, torch.from_numpy(act).to(dev), obs, rew, done)
    scale, offset = np.array(cfg.action_scale[:]), np.array(cfg.action_offset[:])
    tgt = offset[:, None] + scale[:, None] * np.clip(act.T.astype(np.float64), -1.0, 1.0)
    orc = oracle_fleet_from(w, W.Inputs(np.full(n, _abi.AG_MODE_ATT_THRUST, np.uint8), tgt, inp.body, None),
                            s0, m0, e0, seed)
    ocol, _ = O.rollout(world, orc, 1)
    ones = np.ones(n, np.uint32)
    _, o_rew, o_done = O.reach_task(orc.state, goals, ocol, ones, **_params(cfg))
    O.reset(world, orc, (o_done == 1) & (ocol == 0), seed)
    o_obs = O.reach_task(orc.state, goals, ocol, ones, **_params(cfg))[0].T
    np.testing.assert_array_equal(_np(done), o_done)          # max_steps 1: every episode ends
    np.testing.assert_allclose(_np(rew), o_rew, rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(_np(obs), o_obs, atol=2e-6)    # restarted from the reset draw
    fl.close()


def test_reach_full_size_sampled_against_oracle():
    """The bench's task workload (1,048,576 quads, attitude interface, SIE, no
    obstacles) for three task steps with a step limit of 2, so every episode
    ends by time at the second step and restarts from its Philox draw; 2,048
    sampled environments are composed again by the oracle."""
    from paper_2305_16510_gb300.task import ReachEnv
    n, seed = 1 << 20, 1
    rng = np.random.default_rng(seed)
    goals = rng.uniform(-1.0, 1.0, (3, n)).astype(np.float32)
    cfg = _abi.ag_reach_config_default()
    cfg.max_steps = 2
    env = ReachEnv(n, goals=goals, task=cfg, seed=seed)
    env.reset()
    fl = env.fleet
    idx = np.sort(np.random.default_rng(7).choice(n, 2048, replace=False))
    w = W.Workload("reach_full", len(idx), 1, 0, 0, len(idx), 0, 0)
    world = oracle_world(w)
    scale, offset = np.array(cfg.action_scale[:]), np.array(cfg.action_offset[:])
    body = np.tile(np.array([[0.75], [0.007], [0.007], [0.012]], np.float32), (1, len(idx)))
    steps = np.zeros(len(idx), np.uint32)
    ended = 0
    for _ in range(3):
        s0, m0, e0 = _np(fl.state())[:, idx], _np(fl.motors())[:, idx], _np(fl.epoch()).astype(np.uint32)[idx]
        act = rng.uniform(-1.2, 1.2, (n, 4)).astype(np.float32)
        obs, rew, done, _ = env.step(torch.from_numpy(act).cuda())
        g_obs, g_rew, g_done = _np(obs)[idx], _np(rew)[idx], _np(done)[idx]
        tgt = offset[:, None] + scale[:, None] * np.clip(act[idx].T.astype(np.float64), -1.0, 1.0)
        orc = oracle_fleet_from(w, W.Inputs(np.full(len(idx), _abi.AG_MODE_ATT_THRUST, np.uint8), tgt, body, None),
                                s0, m0, e0, seed)
        col, _ = O.rollout(world, orc, 1, env_ids=idx)
        _, o_rew, o_done = O.reach_task(orc.state, goals[:, idx], col, steps + 1, **_params(cfg))
        O.reset(world, orc, (o_done == 1) & (col == 0), seed, env_ids=idx)
        o_obs = O.reach_task(orc.state, goals[:, idx], col, steps + 1, **_params(cfg))[0].T
        np.testing.assert_array_equal(g_done, o_done)
        np.testing.assert_allclose(g_rew, o_rew, rtol=1e-4, atol=1e-4)
        np.testing.assert_allclose(g_obs, o_obs, rtol=1e-4, atol=1e-4)
        np.testing.assert_array_equal(_np(fl.epoch()).astype(np.uint32)[idx], orc.epoch)
        ended += int(g_done.sum())
        steps = np.where(g_done == 1, 0, steps + 1).astype(np.uint32)
    assert ended == len(idx)          # every sampled episode ended at its second step
    env.close()


def test_reach_steps_captured_in_a_cuda_graph_replay_bit_exactly():
    """ag_reach_step issues one kernel on the context's stream and neither
    allocates nor synchronises, so a training loop can capture it in a CUDA
    graph: 8 captured steps replayed 3 times equal 24 direct steps bit for
    bit, collision and time-limit resets included."""
    w = W.Workload("reach_graph", 2048, 4, 1, 8, 2048, 0, 0)
    cfg = _cfg(_abi.AG_MODE_ATT_THRUST, max_steps=5, max_dist=3.0)
    rng = np.random.default_rng(3)
    goals = torch.from_numpy(rng.uniform(-1, 1, (3, w.n_envs)).astype(np.float32)).cuda()
    acts = [torch.from_numpy(rng.uniform(-1, 1, (w.n_envs, 4)).astype(np.float32)).cuda() for _ in range(8)]
    from paper_2305_16510_gb300.fleet import Fleet
    torch.cuda.synchronize()
    results = []
    for use_graph in (False, True):
        side = torch.cuda.Stream()          # capture needs a stream other than the legacy default one
        with torch.cuda.stream(side):
            inp = W.make_inputs(w, 4)
            fl = Fleet(w.n_envs, substeps_per_step=4, integrator=1, n_obstacles=8, seed=4, stream=side)
            fl.set_body(inp.body)
            fl.set_commands(inp.modes, inp.targets)
            fl.set_obstacles(inp.boxes)
            fl.reset(None, 4)
            _abi.ag_reach_begin(fl.ctx, cfg, goals)
            obs = torch.empty((w.n_envs, 13), device=fl.device)
            rew = torch.empty((w.n_envs,), device=fl.device)
            done = torch.empty((w.n_envs,), dtype=torch.uint8, device=fl.device)
            dones = torch.zeros((w.n_envs,), dtype=torch.int32, device=fl.device)
        torch.cuda.synchronize()

        def steps():
            for a in acts:
                _abi.ag_reach_step(fl.ctx, a, obs, rew, done)
                dones.add_(done)

        if use_graph:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=side):
                steps()
            for _ in range(3):
                g.replay()
        else:
            with torch.cuda.stream(side):
                for _ in range(3):
                    steps()
        torch.cuda.synchronize()
        results.append((_np(fl.state()), _np(fl.epoch()), _np(obs), _np(rew), _np(dones)))
        fl.close()
    for a, b in zip(*results):
        np.testing.assert_array_equal(a, b)
    assert results[0][4].sum() > 0                 # episodes ended (and restarted) during the 24 steps
