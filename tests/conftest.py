"""Shared pytest configuration.

Markers: ``gpu`` tests need a CUDA device and the compiled library; every other
test runs on the CPU (the oracle, host logic, the C-ABI symbol table)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled sm_103a library")
    config.addinivalue_line("markers", "slow: long-running full-size check")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle
