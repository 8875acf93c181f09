import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")


@pytest.fixture(scope="session")
def golden_dir():
    return os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="session")
def mdg_lib():
    """Builds (if stale) and loads libmdg.so."""
    from paper_2606_08039_gb300 import build
    build.build_library()
    import paper_2606_08039_gb300 as mdg
    return mdg.lib()


@pytest.fixture(scope="session")
def cuda(mdg_lib):
    """A CUDA device for the GPU parity tests (fails, never skips, without one)."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("the -m gpu tests need a CUDA device")
    torch.cuda.init()
    return torch.device("cuda:0")
