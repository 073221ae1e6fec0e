import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (the GB300 parity tests)")


def pytest_collection_modifyitems(config, items):
    # without a GPU, skip the gpu-marked tests rather than fail them
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(scope="session")
def small():
    from paper_1910_01304_gb300.scenes import workloads
    return workloads.small_scene()


@pytest.fixture(scope="session")
def small4():
    from paper_1910_01304_gb300.scenes import workloads
    return workloads.small_scene(width=4)
