import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built engine library")
    config.addinivalue_line("markers", "slow: large CPU-side cases")
    config.addinivalue_line("markers", "gpu_pending: GPU parity tests of code that has not yet run on a GPU; "
                                       "selected only by -m gpu_pending, skipped without a GPU")


@pytest.fixture(scope="session")
def engine():
    """The engine binding, loaded once; GPU tests only."""
    import paper_2512_12615_gb300 as gx

    return gx
