import os
import sys

import pytest

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def recoil_lib():
    """The built native library (compiled in-tree for sm_103a if missing)."""
    from paper_2306_12141_b300 import build
    build.build()
    import paper_2306_12141_b300 as R
    R.lib()
    return R
