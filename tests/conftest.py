"""Shared pytest configuration.

Tests marked ``gpu`` need a CUDA device and the compiled library; everything else
runs on the CPU (the FP64 oracle, host-side logic, the exported C-ABI symbols).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# every lattice a GPU test closes first has the guard regions around its device buffers
# checked (a write just outside a buffer fails the test that made it)
os.environ.setdefault("LBM_CHECK_GUARDS", "1")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled CUDA library")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.lib()
    return oracle
