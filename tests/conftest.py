import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def lib():
    """The built sm_103a library (skips without a CUDA device)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2003_11679_gb300 as sie
    from paper_2003_11679_gb300 import build
    build.build()
    return sie


@pytest.fixture(scope="session")
def ctx(lib):
    return lib.Context(0)
