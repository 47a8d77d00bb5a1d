import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle

    oracle.load()
    return oracle


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    from tests import parity_log

    lines = parity_log.summary_lines()
    if lines:
        terminalreporter.section("oracle parity: flagged pixels")
        for line in lines:
            terminalreporter.write_line(line)
