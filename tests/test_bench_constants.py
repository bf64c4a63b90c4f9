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


def _tot(c):
    return c["add"] + c["mul"] + c["div"] + c["sqrt"] + c["trans"]


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
