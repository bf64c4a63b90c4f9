"""GB300-native multirotor fleet simulator (arXiv 2305.16510's hot path).

The simulation runs in libaerialgb (hand-written sm_103a CUDA behind the C
ABI of include/ag.h). This package builds that library, binds it with
ctypes (``_abi``, same names as the C entry points) and offers a thin torch
convenience wrapper (``Fleet``). There is no CPU fallback: every entry point
raises if the library is missing.
"""
from . import _abi, build, workloads
from ._abi import AgError

__all__ = ["_abi", "build", "workloads", "AgError", "Fleet"]


def __getattr__(name):
    if name == "Fleet":
        from .fleet import Fleet
        return Fleet
    raise AttributeError(name)
