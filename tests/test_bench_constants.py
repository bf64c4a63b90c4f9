"""The bench's algorithmic work figures are the oracle's operation counts,
its ALU peak comes from the device's own attributes, and its JSON line stays
short enough to be read whole from the tail of the output."""
import json

import oracle as O

import bench
from paper_2305_16510_gb300 import workloads as W


def _tot(c):
    return c["add"] + c["mul"] + c["div"] + c["sqrt"] + c["trans"]


def test_flop_per_vehicle_step_matches_oracle_count():
    w = W.WORKLOADS[bench.WORKLOAD]
    world = O.World(n_envs=1, substeps_per_step=w.substeps_per_step, integrator=w.integrator)
    tot = [_tot(O.count_ops(world, mode, w.n_obstacles)) for mode in w.mode_mix]
    assert abs(sum(tot) / len(tot) - bench.FLOP_PER_VEHICLE_STEP) < 1.0


def test_box_test_flop_matches_oracle_count():
    world = O.World(n_envs=1)
    c0, c1 = O.count_ops(world, W.MODE_WRENCH, 0), O.count_ops(world, W.MODE_WRENCH, 1)
    assert _tot(c1) - _tot(c0) == bench.FLOP_PER_BOX_TEST


def test_alu_peak_from_device_attributes():
    info = {"sm_count": 152, "fp32_lanes_per_sm": 128, "max_sm_clock_khz": 2070000}
    assert abs(bench.alu_peak_tflops(info) - 152 * 128 * 2 * 2.070e9 / 1e12) < 1e-9


def test_mixed_and_paper_shape_flop_figures_match_oracle_count():
    m = W.WORKLOADS["mixed"]
    world = O.World(n_envs=1, substeps_per_step=m.substeps_per_step, integrator=m.integrator, drag=m.drag)
    frac = {4: m.n_quad / m.n_envs, 6: m.n_hexa / m.n_envs, 8: m.n_octo / m.n_envs}
    mixed = sum(f * _tot(O.count_ops(world, W.MODE_BODY_VEL, 0, n_rot)) for n_rot, f in frac.items())
    assert abs(mixed - bench.FLOP_PER_VEHICLE_STEP_MIXED) < 1.0
    p = W.WORKLOADS["paper_shape"]
    world = O.World(n_envs=1, substeps_per_step=p.substeps_per_step, integrator=p.integrator)
    paper = sum(_tot(O.count_ops(world, mode, 0)) for mode in p.mode_mix) / len(p.mode_mix)
    assert abs(paper - bench.FLOP_PER_VEHICLE_STEP_PAPER_SHAPE) < 1.0


def test_depth_flop_figures_match_oracle_count():
    c = O.count_depth_ops()
    assert _tot(c["ray"]) == bench.DEPTH_FLOP_PER_PIXEL
    assert _tot(c["box"]) == bench.DEPTH_FLOP_PER_CAMERA_BOX
    assert _tot(c["pair"]) == bench.DEPTH_FLOP_PER_PIXEL_BOX


def test_adjoint_flop_figures_match_oracle_count():
    a = W.WORKLOADS["adjoint"]
    world = O.World(n_envs=1, substeps_per_step=a.substeps_per_step, integrator=a.integrator)
    fwd, rev = O.count_reverse_ops(world, W.MODE_POSITION, 4)
    assert _tot(fwd) == bench.FLOP_PER_VEHICLE_STEP_ADJ_FWD
    assert _tot(rev) == bench.FLOP_PER_VEHICLE_STEP_ADJ_REV
    # the forward step is the counted vehicle-step plus its loss term: e = p - goal (3 add),
    # w_pos e.e (3 mul + 2 add + 1 mul), w_omega W.W (3 mul + 2 add + 1 mul), two sums (2 add)
    assert _tot(fwd) == _tot(O.count_ops(world, W.MODE_POSITION, 0)) + 17


def _full_result():
    """A result dict shaped like gpu_arm's, with 4-5 significant digits everywhere."""
    rng = [1.3712345e10, 1.3745678e10]
    return {"metric": bench.METRIC, "value": 1.3732214e10, "unit": bench.UNIT, "n_gpus": 1, "steps": 20,
            "warmup": 5, "ms_per_step": 76.358844, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (seeded numpy commands and boxes; Philox initial states)",
            "config": {"workload": bench.WORKLOAD_TEXT, "n_envs": 1048576, "steps_per_call": 1000,
                       "substeps_per_step": 4, "integrator": "rk4", "boxes_per_env": 16, "l2": "x",
                       "parallelism": "replicas x1"},
            "roofline": {"bound": "alu", "achieved": 63.005529, "peak": 80.54784, "unit": "TFLOP/s",
                         "frac": 0.78221252, "traffic": 865260000.0, "kernel": "k", "launch_ms": 76.3,
                         "frac_performed": 0.81234567, "tests_run": 0.04123456,
                         "fma_chain_check": {"packed_tflops": 80.312345, "scalar_tflops": 78.5}},
            "cpu_baseline": {"value": 11817509.8, "unit": bench.UNIT, "cores": 16, "kind": "oracle",
                             "sample": "8192 envs x 15370 steps of the same workload (10.7 s, FP64, 16 threads)",
                             "rows": {"mixed": {"value": 6.3e7}}},
            "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 20},
            "e2e": {"value": 13592003946.19, "unit": bench.UNIT, "h2d_bytes_per_step": 17825792,
                    "d2h_bytes_per_step": 54525952},
            "gpu_launches": 20, "median": 1.3731e10, "range": rng,
            "plain": {"value": 2.78451e9, "fused_over_plain": 4.91234, "hbm_frac": 0.7712345, "range": rng},
            "serving": {"batched": {"value": 7.18234e9, "p50_ms": 12.71234, "p99_ms_median": 148.1234,
                                    "p99_ms_range": [106.123, 200.123], "latency_ms": {"histogram": {}}},
                        "one_per_launch": {"value": 5.96345e9, "p50_ms": 1485.123, "p99_ms": 2049.123},
                        "capacity": {"p99_bound_ms": 250.0, "batched": {"req_per_s": 400.0, "sweep": {}},
                                     "one_per_launch": {"req_per_s": 100.0, "sweep": {}}}},
            "mixed": {"value": 1.10234e11, "alu_frac": 0.80123, "range": [1.09345e11, 1.11234e11]},
            "paper_shape": {"value": 1.14234e11, "alu_frac": 0.74512, "range": [1.13456e11, 1.15678e11]},
            "depth": {"value": 4.32123e6, "alu_frac": 0.51234, "range": [4.3123e6, 4.3589e6]},
            "task": {"value": 1.91234e10, "hbm_frac": 0.79123, "cuda_graph": {"value": 2.07123e10}},
            "adjoint": {"value": 1.46234e10, "alu_frac_record": 0.39123, "alu_frac_backward": 0.55123,
                        "range": [1.45123e10, 1.47345e10]}}


def test_compact_line_is_valid_json_short_and_carries_every_part():
    line = bench.dumps_compact(bench.compact_line(_full_result()))
    assert len(line) < 1450, len(line)          # the tail a reader keeps is 1,500 characters
    d = json.loads(line)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "clocks", "e2e",
              "gpu_launches"):
        assert k in d, k
    assert d["plain"]["fused_over_plain"] > 1
    assert d["serving"]["batched"]["p99_ms"] and d["serving"]["one_per_launch"]["p99_ms"]
    assert d["serving"]["capacity"]["batched"] == 400
    assert d["mixed"]["alu_frac"] and d["paper_shape"]["alu_frac"] and d["roofline"]["fma_chain_tflops"]
    assert d["adjoint"]["alu_bwd"] and d["depth"]["alu_frac"] and d["roofline"]["frac_performed"]
    assert abs(d["value"] - 1.3732214e10) / 1.3732214e10 < 1e-3


def test_dumps_compact_round_trips_numbers():
    x = {"a": 1.23456e10, "b": 7, "c": [0.000123456, -2.5e-7], "d": None, "e": "s", "f": True, "g": 2070.0}
    y = json.loads(bench.dumps_compact(x))
    assert y["b"] == 7 and y["d"] is None and y["e"] == "s" and y["f"] is True and y["g"] == 2070
    assert abs(y["a"] - 1.23456e10) / 1.23456e10 < 1e-3 and abs(y["c"][1] + 2.5e-7) < 1e-12
