"""Shared pytest configuration.

Marker `gpu`: tests that need a CUDA device (run with `-m gpu` on a GB300).
Everything else runs on the CPU (`-m "not gpu"`).
"""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def cuda_available() -> bool:
    try:
        import torch
        return bool(torch.cuda.is_available())
    except Exception:  # pragma: no cover - torch missing
        return False


@pytest.fixture(scope="session")
def cuda_device():
    if not cuda_available():
        pytest.fail("GPU test selected but no CUDA device is visible")
    import torch
    return torch.device("cuda:0")
