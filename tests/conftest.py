"""Test configuration.

Markers: ``gpu`` tests need a CUDA device and call the CUDA library through
its C-ABI; everything else runs on the CPU (oracle pins, graph building and
validation through the C-ABI, multi-process host logic over gloo).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


# Build the CUDA library and the oracle's C checker before any test module
# imports them (both builds are no-ops when up to date).
import __graft_entry__  # noqa: E402

__graft_entry__.build()


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def cuda_device():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")
