import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def cuda_lib():
    """The CUDA library, compiled for sm_103a if any source changed (nvcc cross-compiles without
    a GPU); loading it needs no GPU."""
    from paper_2009_00481_gb300.build import build
    build()
    from paper_2009_00481_gb300 import binding
    return binding.load()
