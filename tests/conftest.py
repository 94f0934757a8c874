import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def hair_small():
    """256 strands x 16 segments x 2 = 8,192 thin tilted triangles, 64x64 rays."""
    from paper_2305_08343_gb300 import scenegen as sg
    return sg.hair(256, 16, False, seed=11), sg.pinhole(64, 64)
