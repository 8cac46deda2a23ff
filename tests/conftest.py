"""Shared pytest configuration: marker registration and seeded problem helpers."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled libgs.so")


@pytest.fixture(scope="session")
def gs_lib():
    """The compiled C-ABI library through its Python binding (GPU tests only)."""
    from paper_2305_08986_gb300 import gs
    return gs
