import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


def pytest_collection_modifyitems(config, items):
    # GPU tests fail loudly (not skip) when the extension is missing on a GPU
    # box; on a machine without a GPU they are deselected by -m "not gpu".
    pass


@pytest.fixture(scope="session")
def rho0_lattice():
    import oracle

    return oracle.rest_density(0.1, 1.0, 0.05)
