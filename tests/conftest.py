import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def scene1():
    from paper_2603_21055_gb300 import synth
    return synth.config1_plane()


@pytest.fixture(scope="session")
def room2():
    """The full 8-keyframe 640x480 room (generated once per session)."""
    from paper_2603_21055_gb300 import synth
    return synth.config2_room()
