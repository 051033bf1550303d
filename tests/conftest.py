import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: large inputs (minutes of host work)")


@pytest.fixture(scope="session", autouse=True)
def _build_host_libs():
    import graphgen
    import oracle
    graphgen.build()
    oracle.build()
    yield


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA library (built in-tree); a GPU test fails loudly when it is missing."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected without a CUDA device")
    import paper_1705_04590_gb300 as bfs
    bfs.load()
    return bfs
