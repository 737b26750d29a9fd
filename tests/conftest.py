import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built library")


@pytest.fixture(scope="session")
def dcrf():
    """The CUDA binding; the library must be built and a GPU present."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device: the GPU tests need one")
    from paper_1608_06192_gb300 import build, _abi
    build.build()
    _abi.lib()
    return _abi
