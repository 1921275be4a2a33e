"""Shared fixtures.  ``-m "not gpu"`` runs the oracle pins, host logic and the
ABI checks on any machine; ``-m gpu`` runs the CUDA parity tests."""
from __future__ import annotations

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer oracle runs")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def plas():
    """The CUDA library (GPU tests only): built if stale, loaded, never a fallback."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2312_13299_gb300 as p
    from paper_2312_13299_gb300 import build as b
    b.build()
    p.load()
    return p
