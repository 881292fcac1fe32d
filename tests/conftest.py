import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built engine library")
    config.addinivalue_line("markers", "slow: large CPU-side cases")


@pytest.fixture(scope="session")
def engine():
    """The engine binding, loaded once; GPU tests only."""
    import paper_2512_12615_gb300 as gx

    return gx


def pytest_collection_finish(session):
    """Before a GPU run: compile the specialised form of the workload and batch programs on
    every host core at once, so each test then loads them from the disk cache instead of
    compiling one after another (a cold cache otherwise costs minutes)."""
    if not any(item.get_closest_marker("gpu") for item in session.items):
        return
    try:
        import torch

        if not torch.cuda.is_available():
            return
    except Exception:
        return
    import paper_2512_12615_gb300 as gx
    from workloads import programs as P

    progs = [P.counting(), P.page_heat(), P.latency()] + list(P.batch_programs())
    gx.precompile(progs, deterministic=True)
