import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# a directory holding a deliberately mutated copy of the oracle package
# (tests/test_oracle_mutants.py only)
if os.environ.get("ORACLE_PY_OVERRIDE"):
    sys.path.insert(0, os.environ["ORACLE_PY_OVERRIDE"])


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.lib()
    return oracle
