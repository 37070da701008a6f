import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def gad():
    """The CUDA library binding; GPU tests fail loudly if it cannot load."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected on a machine without CUDA")
    import paper_1707_09177_gb300 as g
    g.load()
    return g


@pytest.fixture(scope="session")
def golden_table1():
    import json
    with open(os.path.join(ROOT, "tests", "golden", "table1.json")) as f:
        return json.load(f)
