"""Shared pytest set-up: the ``gpu`` marker and import paths.

Tests marked ``gpu`` need a CUDA device and the compiled CUDA library; the rest
run on any CPU.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
TESTS = os.path.dirname(os.path.abspath(__file__))
if TESTS not in sys.path:
    sys.path.insert(0, TESTS)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled CUDA library")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle

    oracle.build_oracle()
    oracle.load()
    return oracle
