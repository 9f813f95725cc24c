"""Shared pytest configuration.

Markers: ``gpu`` marks tests that need a CUDA device (run with ``-m gpu``);
everything else runs on the CPU.  The repository root is put on ``sys.path``
so that ``oracle`` (the CPU reference, test infrastructure) and the package
import without installation.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle
