import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libkpm")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def gpu_lib():
    """The loaded CUDA library; GPU tests fail (not skip) when it is missing."""
    import torch

    assert torch.cuda.is_available(), "GPU test selected but no CUDA device is visible"
    from paper_1105_5481_gb300 import kpm

    return kpm.lib()
