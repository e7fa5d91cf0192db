"""Shared test configuration.

Marker ``gpu``: needs a CUDA device (run with ``-m gpu`` on a GB300).
Everything else runs on the CPU (``-m "not gpu"``).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: test needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def oracle():
    from oracle import oracle as O
    O.build()
    return O


@pytest.fixture(scope="session")
def libgsr_path():
    """Build (if needed) the CUDA library; it must exist for the product path."""
    from paper_2507_15683_gb300 import build
    return build.build()


@pytest.fixture(scope="session")
def gsr(libgsr_path):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a gpu-marked test ran without a CUDA device")
    from paper_2507_15683_gb300 import gsr as G
    return G
