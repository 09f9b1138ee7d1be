import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def litho_lib():
    """The in-tree liblitho.so, built for sm_103a if missing or stale."""
    from paper_2602_15036_gb300 import build as B
    B.build()
    from paper_2602_15036_gb300 import litho
    return litho


@pytest.fixture(scope="session")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")
