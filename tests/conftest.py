import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# frame-server tests run several streams per slot: one hardware queue each
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built liblrvol.so")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def cfg1():
    from paper_1707_01170_gb300.synth import volumes as V
    return V.load_config(1)


@pytest.fixture(scope="session")
def cfg1_oracle(cfg1):
    from oracle.oracle import Oracle
    return Oracle(cfg1)
