import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: full-size parity cases")


@pytest.fixture(scope="session")
def ssamg_lib():
    """The CUDA library, built in-tree if it is missing (nvcc cross-compiles
    for sm_103a without a GPU)."""
    from paper_2205_14273_gb300 import ssamg as S
    if not os.path.exists(S.LIB_PATH):
        from paper_2205_14273_gb300 import build_lib
        build_lib.build()
    return S
