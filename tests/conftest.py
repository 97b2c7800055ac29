import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running test")


@pytest.fixture(scope="session")
def ep_lib():
    """The CUDA library's Python binding; on a machine with a GPU a missing
    library is an error, never a fallback."""
    from paper_2308_01651_gb300 import ep
    return ep


@pytest.fixture(scope="session", autouse=True)
def _cuda_library_built():
    """Builds the CUDA library in-tree when it is missing (nvcc compiles for
    sm_103a without a GPU), so that the host-side checks of the C ABI run from
    a clean checkout; building is not using it, and the GPU tests need it
    anyway."""
    from paper_2308_01651_gb300 import build as B
    from paper_2308_01651_gb300 import ep
    if not os.path.exists(ep.LIB_PATH):
        B.build()
