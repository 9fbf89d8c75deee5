import os
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built librgf.so")
    config.addinivalue_line("markers", "slow: long-running (full-size workloads)")


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


HAS_GPU = _has_gpu()


def pytest_collection_modifyitems(config, items):
    if HAS_GPU:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(scope="session")
def rgflib():
    """The ctypes binding; builds librgf.so in-tree first if it is missing."""
    lib = ROOT / "paper_1107_5300_gb300" / "librgf.so"
    if not lib.exists():
        from paper_1107_5300_gb300.build import build
        build()
    from paper_1107_5300_gb300 import rgf
    return rgf
