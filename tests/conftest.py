"""Shared pytest configuration.

Tests marked ``gpu`` need a CUDA device and the CUDA library; everything else
runs on the CPU (the oracle and its pins, host logic, the C-ABI exports).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled CUDA library")
    config.addinivalue_line("markers", "slow: long-running statistical check")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.lib()
    return oracle
