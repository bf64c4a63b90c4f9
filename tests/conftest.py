import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# (test, quantity, measured, bound) of every within_tolerance check of the session
_TOLERANCES: list[dict] = []


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels through the C-ABI)")


@pytest.fixture
def within_tolerance(request):
    """check(quantity, measured, bound): asserts measured <= bound and records
    both, so a run with AG_TOLERANCE_REPORT=<file> writes every parity test's
    measured error beside its bound (the margin each bound leaves)."""
    def check(quantity: str, measured: float, bound: float) -> None:
        measured = float(measured)
        _TOLERANCES.append({"test": request.node.name, "quantity": quantity, "measured": measured,
                            "bound": float(bound)})
        assert measured <= bound, f"{quantity}: {measured:.3g} > {bound:.3g}"
    return check


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("AG_TOLERANCE_REPORT")
    if path and _TOLERANCES:
        with open(path, "w") as f:
            json.dump(_TOLERANCES, f, indent=1)
