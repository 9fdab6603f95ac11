import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")


@pytest.fixture(scope="session")
def oracle():
    from oracle import oracle as O
    O.build()
    return O


def pytest_terminal_summary(terminalreporter):
    """Print what the parity tests measured (pair counts, error figures)."""
    try:
        from tests.gpu_cases import REPORT
    except ImportError:
        return
    if REPORT:
        terminalreporter.section("parity report")
        for line in REPORT:
            terminalreporter.write_line(line)
