"""The continuous-batching server (ag_server_*): results, batching, admission.

Every request's final state must be bit-identical whether it runs alone, in a
mix of uneven requests that arrive while it runs, or with one request per
launch; a served request must match the FP64 oracle and the context path
(ag_step) on the same inputs; admission must keep the slab within its HBM
budget; waits are bounded.
"""
import time

import numpy as np
import pytest
import torch

import oracle as O
from harness import max_state_errors
from paper_2305_16510_gb300 import _abi
from paper_2305_16510_gb300 import workloads as W

pytestmark = pytest.mark.gpu
N_POOL = 40000


@pytest.fixture(scope="module")
def pool():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2305_16510_gb300 import build
    build.build()
    from paper_2305_16510_gb300.serving import RequestPool
    w = W.Workload("pool", N_POOL, 4, 1, 32, N_POOL, 0, 0,
                   mode_mix=(W.MODE_POSITION, W.MODE_BODY_VEL, W.MODE_ATT_THRUST))
    inp = W.make_inputs(w, 2024)
    return RequestPool(inp.modes, inp.targets, inp.boxes.reshape(32 * 10, N_POOL)), inp


def _server(**kw):
    from paper_2305_16510_gb300.serving import Server
    return Server(**kw)


def test_request_is_bit_identical_alone_in_a_mix_and_one_per_launch(pool):
    rp, _ = pool
    target = dict(n_envs=3000, n_steps=180, n_obstacles=8, seed=11, offset=100)
    with _server(max_active=64, chunk_steps=50) as s:
        st_alone, ep_alone, _ = s.wait(s.submit(rp.request(**target)))
    rng = np.random.default_rng(3)
    with _server(max_active=64, chunk_steps=50) as s:
        ids = []
        for k in range(14):
            if k == 5:
                ids.append(("target", s.submit(rp.request(**target))))
            n = int(rng.integers(256, 9000))
            ids.append(("other", s.submit(rp.request(n, int(rng.integers(50, 400)), int(rng.choice([0, 8, 32])),
                                                     seed=100 + k, offset=int(rng.integers(0, N_POOL - n))))))
            time.sleep(0.002)          # arrivals while earlier requests run
        res = {}
        for tag, rid in ids:
            res[rid] = s.wait(rid)
        st_mix, ep_mix, _ = res[[rid for tag, rid in ids if tag == "target"][0]]
        stats = s.stats()
        assert stats.completed == len(ids)
        assert stats.launches < sum(1 for _ in ids) * 8     # requests shared launches
    np.testing.assert_array_equal(st_mix, st_alone)
    np.testing.assert_array_equal(ep_mix, ep_alone)
    with _server(max_active=1, chunk_steps=50) as s:
        st_one, ep_one, _ = s.wait(s.submit(rp.request(**target)))
    np.testing.assert_array_equal(st_one, st_alone)
    np.testing.assert_array_equal(ep_one, ep_alone)


def test_tiny_and_odd_requests_are_bit_identical_alone_and_in_a_mix(pool):
    """Requests smaller than a block or a warp, odd box counts (a padded pair)
    and unaligned pool offsets: each result alone equals its result in a mix."""
    rp, _ = pool
    shapes = [(1, 60, 0), (2, 75, 1), (31, 50, 3), (33, 120, 8), (129, 90, 32)]
    reqs = [dict(n_envs=n, n_steps=h, n_obstacles=o, seed=500 + k, offset=17 * k + 3)
            for k, (n, h, o) in enumerate(shapes)]
    alone = []
    with _server(max_active=8, chunk_steps=50) as s:
        for r in reqs:
            st, ep, _ = s.wait(s.submit(rp.request(**r)))
            alone.append((st, ep))
    with _server(max_active=8, chunk_steps=50) as s:
        ids = [s.submit(rp.request(**r)) for r in reqs]
        mixed = [s.wait(i)[:2] for i in ids]
    for (n, h, o), (a_st, a_ep), (m_st, m_ep) in zip(shapes, alone, mixed):
        assert a_st.shape == (13, n) and np.isfinite(a_st).all()
        np.testing.assert_array_equal(m_st, a_st, err_msg=f"n={n} boxes={o}")
        np.testing.assert_array_equal(m_ep, a_ep)


def test_served_request_matches_the_oracle(pool):
    rp, inp = pool
    n, steps, seed, off = 600, 60, 5, 1234
    with _server(max_active=8, chunk_steps=25) as s:
        st, ep, lat = s.wait(s.submit(rp.request(n, steps, 0, seed=seed, offset=off)))
    assert lat > 0
    world = O.World(n_envs=n, substeps_per_step=4, integrator=O.INTEG_RK4)
    fl = O.make_fleet(world, modes=inp.modes[off:off + n], targets=inp.targets[:, off:off + n].astype(np.float64),
                      seed=seed)
    O.reset(world, fl, None, seed)
    O.rollout(world, fl, steps, n_threads=8)
    dp, _, dang, _ = max_state_errors(st, fl.state)
    scale = 1.0 + np.max(np.abs(fl.state[0:3]), axis=0)
    assert np.all(dp <= 1e-4 * scale), dp.max()
    assert dang.max() <= 2e-4
    assert np.all(ep == 1)


def test_served_request_matches_the_context_path(pool, monkeypatch):
    """A served request against the same fleet stepped through the context
    (two 50-step ag_step calls), in both thread orders of the context. The
    server's kernel, the fused kernel's branching loop (identity order) and
    its loops compiled per command mode (grouped order) are separate
    programs; every fused multiply-add of the step is explicit and nothing
    else is contracted, so all of them must agree bit for bit."""
    rp, inp = pool
    from harness import gpu_fleet
    n, seed, off = 2500, 9, 5000
    with _server(max_active=8, chunk_steps=50) as s:
        st, ep, _ = s.wait(s.submit(rp.request(n, 100, 32, seed=seed, offset=off)))
    w = W.Workload("ctx", n, 4, 1, 32, n, 0, 0)
    sub = W.Inputs(inp.modes[off:off + n].copy(), np.ascontiguousarray(inp.targets[:, off:off + n]),
                   W.body(w, np.random.default_rng(0)), np.ascontiguousarray(inp.boxes[:, :, off:off + n]))
    for order in ("identity", "grouped"):
        if order == "identity":
            monkeypatch.setenv("AG_FUSED_ORDER", "identity")
        else:
            monkeypatch.delenv("AG_FUSED_ORDER")
        fl = gpu_fleet(w, sub, seed)
        fl.reset(None, seed)
        fl.step(50)
        fl.step(50)
        st_ctx = fl.state().cpu().numpy()
        ep_ctx = fl.epoch().cpu().numpy().astype(np.uint32)
        fl.close()
        assert np.mean(ep_ctx > 1) > 0.01                  # collisions happened
        np.testing.assert_array_equal(ep, ep_ctx, err_msg=order)
        np.testing.assert_array_equal(st, st_ctx, err_msg=order)


def test_admission_stays_within_the_hbm_budget(pool):
    rp, _ = pool
    budget = 96 << 20
    rng = np.random.default_rng(4)
    peak = 0
    with _server(max_active=256, chunk_steps=20, hbm_budget_bytes=budget) as s:
        ids = [s.submit(rp.request(int(rng.integers(5000, 20000)), 100, 32, seed=k, offset=0)) for k in range(24)]
        done = 0
        while done < len(ids):
            st = s.stats()
            peak = max(peak, st.hbm_used_bytes)
            assert st.hbm_used_bytes <= budget
            done = st.completed
            time.sleep(0.001)
        for rid in ids:
            s.wait(rid, want_state=False)
    assert peak > budget // 4          # the budget, not the slot count, limited admission


def test_bounded_wait_and_invalid_requests(pool):
    rp, _ = pool
    with _server(max_active=4, chunk_steps=100) as s:
        rid = s.submit(rp.request(N_POOL, 3000, 32, seed=1))
        with pytest.raises(_abi.AgError) as e:
            s.wait(rid, timeout_s=0.0005)
        assert e.value.status == _abi.AG_ERR_TIMEOUT
        s.wait(rid, timeout_s=600)       # still there, completes
        for n_bad in (0, _abi.AG_MAX_ENVS + 1):   # counts are checked before any array is read
            bad = rp.request(10, 10, 0, seed=1)
            bad.n_envs = n_bad
            with pytest.raises(_abi.AgError) as e:
                s.submit(bad)
            assert e.value.status == _abi.AG_ERR_INVALID
    with _server(max_active=4, chunk_steps=10, hbm_budget_bytes=8 << 20) as s:
        with pytest.raises(_abi.AgError) as e:
            s.submit(rp.request(N_POOL, 10, 32, seed=1))
        assert e.value.status == _abi.AG_ERR_OOM
