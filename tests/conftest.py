import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# measured figures that tests record for the run's summary (per-replica errors
# and the like): printed at the end of the session even when the tests pass
_REPORT = []


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture
def report():
    """report(line): add a line to the session's measurement summary."""
    return _REPORT.append


def pytest_terminal_summary(terminalreporter):
    if _REPORT:
        terminalreporter.section("measurements recorded by the tests")
        for line in _REPORT:
            terminalreporter.write_line(line)
