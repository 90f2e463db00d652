import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session", autouse=True)
def _built_oracle():
    """Compile the oracle's C part once per session if it is missing."""
    lib = os.path.join(ROOT, "oracle", "libsofa_oracle.so")
    if not os.path.exists(lib):
        import __graft_entry__ as g
        g.build_oracle()
    yield
