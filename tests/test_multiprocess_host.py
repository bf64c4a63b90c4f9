"""Multi-process host logic of bench.py on CPU (gloo, world size 2).

The environments are independent, so the bench runs one full-size replica
per rank with no collective on the data path; what the ranks share is the
barrier around the timed region and the maximum of their times. These tests
run that logic in two gloo processes and check the reference arm's rule that
ranks other than 0 do no work.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys, time
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
world, rank, _ = bench.dist_env()
dist.init_process_group("gloo", rank=rank, world_size=world)
t0 = time.perf_counter()
if rank == 1:
    time.sleep(0.3)                       # the slow rank
bench.barrier(world)                      # rank 0 waits here for rank 1
waited = time.perf_counter() - t0
slowest = bench.max_over_ranks(float(rank + 1) * 1.5, world)
rate = bench.whole_job_rate(1000.0, world, slowest)
dist.destroy_process_group()
print(json.dumps({"rank": rank, "waited": waited, "slowest": slowest, "rate": rate}))
"""


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_ranks(code: str, world: int = 2, extra_args=()):
    port = _free_port()
    procs = []
    for rank in range(world):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code, ROOT, *extra_args], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(out)
    return outs


def test_barrier_and_max_over_ranks_with_gloo():
    outs = [json.loads(o.strip().splitlines()[-1]) for o in _run_ranks(WORKER)]
    by_rank = {o["rank"]: o for o in outs}
    assert set(by_rank) == {0, 1}
    assert by_rank[0]["waited"] >= 0.25                      # the barrier held rank 0 for rank 1
    assert all(o["slowest"] == 3.0 for o in outs)            # max of 1.5 and 3.0 on every rank
    assert all(abs(o["rate"] - 1000.0 * 2 / 3.0) < 1e-9 for o in outs)


REFERENCE = r"""
import sys, time
sys.path.insert(0, sys.argv[1])
import bench
sys.argv = ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"]
t0 = time.perf_counter()
bench.main()
print("elapsed", time.perf_counter() - t0)
"""


def test_reference_arm_runs_on_rank_zero_only():
    # rank 1 of a 2-rank job prints no JSON line and returns at once
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    p = subprocess.run([sys.executable, "-c", REFERENCE, ROOT], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1 and lines[0].startswith("elapsed")
    assert float(lines[0].split()[1]) < 5.0


def test_whole_job_rate_is_weak_scaling():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(1e6, 1, 2.0) == 5e5
    assert bench.whole_job_rate(1e6, 4, 2.0) == 2e6          # 4 replicas, each 1e6 units, slowest 2 s
