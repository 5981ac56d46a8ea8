import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.fixture(scope="session")
def golden():
    return read_golden


def pytest_terminal_summary(terminalreporter):
    """The per-step parity counts of the GPU tests (steps replayed, steps the
    rounding bound forces, agreement with the oracle's selection from the
    GPU's own iterates), printed even under -q."""
    try:
        from stepcheck import REPORT
    except ImportError:
        return
    if REPORT:
        terminalreporter.write_sep("-", "per-step parity")
        for line in REPORT:
            terminalreporter.write_line(line)
