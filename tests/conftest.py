import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long CPU-only check, excluded from the default CPU suite")


_ERRORS = []


def record_error(case: str, **values):
    """Collect a measured error (written to $LGF_ERROR_LOG at session end)."""
    _ERRORS.append({"case": case, **{k: float(v) for k, v in values.items()}})


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("LGF_ERROR_LOG")
    if path and _ERRORS:
        import json
        with open(path, "w") as fh:
            for e in _ERRORS:
                fh.write(json.dumps(e) + "\n")
