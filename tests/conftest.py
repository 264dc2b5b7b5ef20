import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 and the CUDA library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def bfi():
    """The CUDA library's Python binding (built in-tree on first use)."""
    import __graft_entry__
    __graft_entry__._build_module().build()
    import paper_1803_07560_gb300 as mod
    return mod
