import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: slower CPU test")


@pytest.fixture(scope="session")
def golden_dir():
    return GOLDEN


@pytest.fixture(scope="session")
def Mr_5_25():
    from oracle.fc_tables import fc_matrix
    return fc_matrix(5, 25, table_dir=GOLDEN)


@pytest.fixture(scope="session")
def Mr_7_33():
    from oracle.fc_tables import fc_matrix
    return fc_matrix(7, 33, table_dir=GOLDEN)
