import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 (sm_103a) and the compiled CUDA library")


@pytest.fixture(scope="session")
def small():
    from paper_1204_6367_gb300 import inputs
    return inputs.small_problem()


@pytest.fixture(scope="session")
def torso():
    from paper_1204_6367_gb300 import inputs
    return inputs.torso_problem()
