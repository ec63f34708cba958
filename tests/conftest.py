import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


@pytest.fixture(scope="session")
def h2mech():
    import synth
    return synth.h2_air_mechanism(0)


@pytest.fixture(scope="session")
def hcmech():
    import synth
    return synth.hydrocarbon_mechanism(0)
