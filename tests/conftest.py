import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def room():
    from paper_2507_04021_gb300 import inputs
    return inputs.room_scene()


@pytest.fixture(scope="session")
def office():
    from paper_2507_04021_gb300 import inputs
    return inputs.office_scene()
