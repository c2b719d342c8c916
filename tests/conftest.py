import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libhv.so")
    config.addinivalue_line("markers", "slow: oracle runs of more than a few seconds")


@pytest.fixture(autouse=True)
def _release_device_buffers():
    """Device frames handed to the library stay alive until the test has ended
    and the device is idle (the library copies them on its own streams)."""
    yield
    from tests._util import release_device_buffers
    release_device_buffers()
