"""Shared pytest setup: the ``gpu`` marker, import paths, and the optional parity report."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("CDP_PARITY_REPORT")
    if not path:
        return
    import parity_report

    if parity_report.RESULTS:
        with open(path, "w") as f:
            json.dump(parity_report.RESULTS, f, indent=1, sort_keys=True)
