import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libjbp.so")


@pytest.fixture(scope="session")
def oracle():
    from oracle import oracle as O
    O.build()
    return O


@pytest.fixture(scope="session")
def jbp_lib():
    """The CUDA library, built in-tree if missing (nvcc cross-compiles without a GPU)."""
    from paper_2605_26580_gb300 import build as B
    B.build()
    from paper_2605_26580_gb300 import jbp
    jbp.lib()
    return jbp
