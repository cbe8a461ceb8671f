import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: full-size cases (tens of seconds on the CPU oracle)")


@pytest.fixture(scope="session")
def cfg1():
    from paper_1603_08161_b300 import synth
    return synth.config1()


@pytest.fixture(scope="session")
def cfg2():
    from paper_1603_08161_b300 import synth
    return synth.config2()
