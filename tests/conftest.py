import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled pmplus library")


@pytest.fixture(scope="session")
def native():
    """The compiled CUDA library through its Python binding (GPU tests only)."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_09840_gb300 import native as nat

    nat.load()  # raises if the extension is missing: no fallback
    return nat
