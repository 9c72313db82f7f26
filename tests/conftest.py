import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU oracle work")


@pytest.fixture(scope="session")
def toy_oracle():
    from oracle import oracle as O
    o = O.Oracle(7, O.toy_params())
    yield o
    o.close()


@pytest.fixture(scope="session")
def real_oracle():
    from oracle import oracle as O
    o = O.Oracle(11)
    yield o
    o.close()
