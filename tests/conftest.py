import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built extension")
    config.addinivalue_line("markers", "slow: long-running oracle cases")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def ctx():
    """A library context on cuda:0 (GPU tests only)."""
    from paper_1201_1548_gb300.build import build
    build()
    import paper_1201_1548_gb300 as bs
    c = bs.Context(0)
    yield c
    c.close()
