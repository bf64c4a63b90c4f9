"""The bench's per-vehicle-step FLOP figure is the oracle's operation count."""
import oracle as O

import bench
from paper_2305_16510_gb300 import workloads as W


def test_flop_per_vehicle_step_matches_oracle_count():
    w = W.WORKLOADS[bench.WORKLOAD]
    world = O.World(n_envs=1, substeps_per_step=w.substeps_per_step, integrator=w.integrator)
    tot = []
    for mode in w.mode_mix:
        c = O.count_ops(world, mode, w.n_obstacles)
        tot.append(c["add"] + c["mul"] + c["div"] + c["sqrt"] + c["trans"])
    assert abs(sum(tot) / len(tot) - bench.FLOP_PER_VEHICLE_STEP) < 1.0


def test_alu_peak_from_unit_counts():
    assert abs(bench.ALU_PEAK_TFLOPS - 152 * 128 * 2 * 2.070e9 / 1e12) < 1e-9
