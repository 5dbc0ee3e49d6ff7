import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def orc():
    # FIC_ORACLE_DIR names a folder holding a copy of the oracle package with a
    # planted mistake (tests/test_oracle_mutants.py runs the pins against it)
    alt = os.environ.get("FIC_ORACLE_DIR")
    if alt:
        sys.path.insert(0, alt)
    import oracle

    if alt:
        assert os.path.dirname(os.path.dirname(os.path.abspath(oracle.__file__))) == os.path.abspath(alt)
    oracle.build()
    return oracle
