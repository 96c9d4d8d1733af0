import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running (full-size workloads)")


@pytest.fixture(scope="session", autouse=True)
def _built():
    """Builds the generator, the oracle and the library once per session (no-op when fresh)."""
    import __graft_entry__ as ge

    ge.build_all(import_package=False)
    yield


def has_gpu():
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False
