import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: oracle cases that take more than ~20 s on the CPU")


@pytest.fixture(scope="session")
def n10():
    from paper_2606_04186_gb300 import synth
    return synth.system_inputs("n10")
