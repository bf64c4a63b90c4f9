"""Contexts driven from several host threads at once.

Each context owns its buffers and its stream. The library's process-wide
state (cached occupancy figures, the per-device shared-memory attribute of
the fused kernel, the build lock) is shared. Four threads create, step,
reset, render and destroy their own contexts concurrently, on their own
streams, and every result must be bit-identical to the same work done one
context after another.
"""
import threading

import numpy as np
import pytest
import torch

from harness import gpu_fleet
from paper_2305_16510_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CONFIGS = [
    W.Workload("thr_rk4_boxes", 3000, 4, 1, 8, 3000, 0, 0),                  # fused step with box staging
    W.Workload("thr_mixed", 2500, 1, 0, 0, 1000, 1000, 500, drag=0.1),       # quad / hexa / octo, no boxes
    W.Workload("thr_odd_boxes", 4096, 2, 1, 3, 4096, 0, 0),                  # odd box count (padded pair)
    W.Workload("thr_many_boxes", 1000, 1, 0, 16, 1000, 0, 0),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2305_16510_gb300 import build
    build.build()


def _run_context(w, seed):
    """Reset, fused and unfused steps, a masked reset and a depth render on a
    context of its own, on a stream of its own; returns the results on the host."""
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        inp = W.make_inputs(w, seed)
        fl = gpu_fleet(w, inp, seed)
        fl.reset(None, seed)
        for r in range(4):
            fl.step(10)
            fl.step_plain(1)
            fl.reset(W.reset_mask(w.n_envs, 0.05, np.random.default_rng(seed + r)), seed + r)
        fl.step(10)
        col, ids = fl.events()
        out = {"state": fl.state().cpu().numpy(), "motors": fl.motors().cpu().numpy(),
               "epoch": fl.epoch().cpu().numpy(), "collided": col.cpu().numpy(),
               "resets": np.sort(ids.cpu().numpy())}
        if w.n_obstacles:
            out["depth"] = fl.render_depth(40, 24, 1.5, 10.0, env_ids=np.arange(0, w.n_envs, 97)).cpu().numpy()
        fl.close()
    return out


def test_contexts_in_concurrent_threads_match_sequential_runs():
    seeds = [31 + k for k in range(len(CONFIGS))]
    sequential = [_run_context(w, s) for w, s in zip(CONFIGS, seeds)]
    for _ in range(3):           # repeated, to give interleavings a chance
        results, errors = [None] * len(CONFIGS), []

        def run(k):
            try:
                results[k] = _run_context(CONFIGS[k], seeds[k])
            except BaseException as e:       # re-raised below, on the test's thread
                errors.append(e)

        threads = [threading.Thread(target=run, args=(k,)) for k in range(len(CONFIGS))]
        for t in threads:
            t.start()
        for t in threads:
            t.join(timeout=600)
        assert not any(t.is_alive() for t in threads)
        if errors:
            raise errors[0]
        for k, (a, b) in enumerate(zip(sequential, results)):
            assert a.keys() == b.keys()
            for key in a:
                np.testing.assert_array_equal(a[key], b[key], err_msg=f"{CONFIGS[k].name}: {key}")
