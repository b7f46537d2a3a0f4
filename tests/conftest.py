import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: oracle cases that take more than a few seconds")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def mdp():
    """The package with libmdp.so built in-tree (nvcc cross-compiles without a GPU)."""
    from paper_2103_12172_gb300 import _build
    _build.build()
    import paper_2103_12172_gb300 as pkg
    return pkg
