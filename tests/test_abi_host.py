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
