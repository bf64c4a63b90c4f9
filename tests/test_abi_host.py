"""Host-side checks of the C-ABI library (no GPU: no compute calls).

The library must build, load, export every function include/ag.h declares,
and reject invalid configurations before touching the device.
"""
import os
import re
import subprocess

import pytest

from paper_2305_16510_gb300 import _abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ag_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _abi.lib()


def test_library_exports_every_declared_symbol(lib):
    declared = declared_functions()
    assert {"ag_create", "ag_step", "ag_reset", "ag_get_state", "ag_set_commands"} <= declared
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ag_[a-z0-9_]+)", out))
    assert declared <= exported, declared - exported
    # the binding wraps exactly the declared entry points
    assert declared == set(_abi.SIGNATURES)


def test_abi_version_and_defaults(lib):
    header = open(os.path.join(ROOT, "include", "ag.h")).read()
    assert "#define AG_MAX_ENVS (1u << 28)" in header and _abi.AG_MAX_ENVS == 1 << 28
    assert f"#define AG_MAX_OBSTACLES {_abi.AG_MAX_OBSTACLES}" in header
    assert f"#define AG_ABI_VERSION {_abi.ABI_VERSION}" in header
    assert _abi.ag_abi_version() == _abi.ABI_VERSION
    c = _abi.ag_config_default()
    assert c.n_envs == 1024 and c.n_quad == 1024 and c.substeps_per_step == 1
    assert abs(c.dt - 0.01) < 1e-9 and abs(c.u_max - 5.0) < 1e-9 and abs(c.motor_tau - 0.03) < 1e-9
    assert [round(x, 6) for x in c.kx] == [2, 2, 3]
    assert [round(x, 6) for x in c.kR] == [1.2, 1.2, 0.6]


@pytest.mark.parametrize("field,value,msg", [
    ("n_envs", 0, "n_envs"),
    ("n_envs", (1 << 28) + 1, "AG_MAX_ENVS"),   # larger fleets would overflow 32-bit field indices
    ("substeps_per_step", 0, "substeps_per_step"),
    ("substeps_per_step", 65537, "substeps_per_step"),
    ("record_every", 65537, "record_every"),
    ("integrator", 7, "integrator"),
    ("n_obstacles", 65, "n_obstacles"),
    ("n_quad", 5, "n_quad + n_hexa + n_octo"),
    ("dt", 0.0, "dt"),
    ("u_max", -1.0, "u_max"),
    ("mass", 0.0, "mass"),
])
def test_invalid_config_rejected_before_device_use(lib, field, value, msg):
    c = _abi.ag_config_default()
    setattr(c, field, value)
    with pytest.raises(_abi.AgError) as e:
        _abi.ag_create(c)
    assert e.value.status == _abi.AG_ERR_INVALID
    assert msg in str(e.value)


def test_null_context_is_invalid(lib):
    assert lib.ag_step(None, 1) == _abi.AG_ERR_INVALID
    assert lib.ag_reset(None, None, 1) == _abi.AG_ERR_INVALID
    assert lib.ag_destroy(None) == _abi.AG_OK


def test_header_is_plain_c():
    # the boundary carries no torch or C++ types
    src = open(os.path.join(ROOT, "include", "ag.h")).read()
    for bad in ("torch", "at::", "std::", "Tensor", "template"):
        assert bad not in src
    r = subprocess.run(["gcc", "-std=c99", "-fsyntax-only", "-x", "c", os.path.join(ROOT, "include", "ag.h")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_measure_fp32_peak_rejects_bad_arguments(lib):
    # argument checks come before any CUDA call, so they run without a GPU
    for kw in ({"iters": 0}, {"iters": 1000001}, {"reps": 0}, {"reps": 101}):
        with pytest.raises(_abi.AgError) as e:
            _abi.ag_measure_fp32_peak(**kw)
        assert e.value.status == _abi.AG_ERR_INVALID
    assert lib.ag_measure_fp32_peak(None, 10, 1, None) == _abi.AG_ERR_INVALID
    assert b"out is NULL" in lib.ag_last_error(None)


def _config_is_valid(c) -> bool:
    """The rules include/ag.h states for ag_config, written out independently."""
    import math
    finite_pos = lambda x: math.isfinite(x) and x > 0
    return (1 <= c.n_envs <= (1 << 28) and 1 <= c.substeps_per_step <= 65536 and c.integrator <= 1
            and c.n_obstacles <= 64 and c.n_quad + c.n_hexa + c.n_octo == c.n_envs and c.record_every <= 65536
            and finite_pos(c.dt) and c.motor_tau >= 0 and c.drag >= 0 and c.sphere_r >= 0 and c.u_max > 0
            and c.arm > 0 and c.k_yaw > 0 and c.mass > 0 and all(x > 0 for x in c.inertia))


def test_config_validation_follows_the_documented_rules(lib):
    """Random valid configurations with at most one documented rule broken:
    ag_create refuses exactly the broken ones (AG_ERR_INVALID, before any
    device call). Valid ones get to the device step: without a GPU that is
    AG_ERR_CUDA ("no CUDA device"); with one, a small context is created and
    destroyed."""
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies
    pos = st.sampled_from([1e-3, 0.01, 0.13, 0.5, 5.0])
    breaks = {
        None: lambda c: None,
        "n_envs 0": lambda c: setattr(c, "n_envs", 0),
        "n_envs above AG_MAX_ENVS": lambda c: setattr(c, "n_envs", (1 << 28) + 1),
        "substeps 0": lambda c: setattr(c, "substeps_per_step", 0),
        "substeps above 65536": lambda c: setattr(c, "substeps_per_step", 65537),
        "integrator 2": lambda c: setattr(c, "integrator", 2),
        "65 boxes": lambda c: setattr(c, "n_obstacles", 65),
        "type counts": lambda c: setattr(c, "n_quad", c.n_quad + 1),
        "record_every": lambda c: setattr(c, "record_every", 65537),
        "dt 0": lambda c: setattr(c, "dt", 0.0),
        "dt inf": lambda c: setattr(c, "dt", float("inf")),
        "dt nan": lambda c: setattr(c, "dt", float("nan")),
        "tau < 0": lambda c: setattr(c, "motor_tau", -0.01),
        "drag < 0": lambda c: setattr(c, "drag", -0.1),
        "radius < 0": lambda c: setattr(c, "sphere_r", -0.2),
        "u_max 0": lambda c: setattr(c, "u_max", 0.0),
        "arm nan": lambda c: setattr(c, "arm", float("nan")),
        "k_yaw < 0": lambda c: setattr(c, "k_yaw", -0.016),
        "mass 0": lambda c: setattr(c, "mass", 0.0),
        "inertia nan": lambda c: c.inertia.__setitem__(1, float("nan")),
    }

    @hyp.settings(max_examples=150, deadline=None, derandomize=True)
    @hyp.given(n=st.sampled_from([1, 7, 33, 4096]), sub=st.sampled_from([1, 4, 65536]), integ=st.sampled_from([0, 1]),
               obs=st.sampled_from([0, 3, 64]), mixed=st.booleans(), rec=st.sampled_from([0, 32, 65536]),
               dt=pos, tau=st.sampled_from([0.0, 0.03]), drag=st.sampled_from([0.0, 0.1]), umax=pos, arm=pos,
               kyaw=pos, mass=pos, which=st.sampled_from([None] * 10 + list(breaks)))  # ~1/3 valid
    def check(n, sub, integ, obs, mixed, rec, dt, tau, drag, umax, arm, kyaw, mass, which):
        c = _abi.ag_config_default()
        c.n_envs, c.substeps_per_step, c.integrator, c.n_obstacles, c.record_every = n, sub, integ, obs, rec
        c.n_hexa, c.n_octo = (n // 3, n // 4) if mixed else (0, 0)
        c.n_quad = n - c.n_hexa - c.n_octo
        c.dt, c.motor_tau, c.drag, c.u_max, c.arm, c.k_yaw, c.mass = dt, tau, drag, umax, arm, kyaw, mass
        breaks[which](c)
        valid = _config_is_valid(c)
        assert valid == (which is None), which          # the rule list itself agrees with the break
        try:
            ctx = _abi.ag_create(c)
        except _abi.AgError as e:
            expect = _abi.AG_ERR_CUDA if valid else _abi.AG_ERR_INVALID
            assert e.status == expect, (which, e.status, str(e))
            return
        assert valid, which
        _abi.ag_destroy(ctx)

    check()


def test_step_sources_compile_without_implicit_contraction():
    """Every file that compiles the per-vehicle step (the fused kernels and
    their per-mode loops, the unfused stages, the serving kernel, the task
    step) writes its fused multiply-adds out and is compiled with
    -fmad=false, so that each compiled copy rounds as the source says and
    the copies agree bit for bit; a new file that includes the step's
    headers must join them."""
    import os
    import re
    from paper_2305_16510_gb300 import build
    for src in build.CUDA_SOURCES:
        text = open(os.path.join(build.CSRC, src)).read()
        includes = set(re.findall(r'#include "([^"]+)"', text))
        runs_step = "fleet_sim.cuh" in includes or ("fleet_device.cuh" in includes and "simulate" in text)
        if runs_step:
            assert src in build.NO_CONTRACTION, src
    assert {"fleet_kernels.cu", "serve.cu", "task.cu"} <= build.NO_CONTRACTION
