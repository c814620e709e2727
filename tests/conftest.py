import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU oracle test")


LIB = os.path.join(ROOT, "paper_2602_16591_gb300", "libpswf_ewald.so")


def require_library():
    """The CUDA library's Python binding, for test modules that call the library.

    On a machine without a GPU and without the built library the calling module is skipped (the
    oracle's own tests need neither).  With a GPU present a missing library is an error: there is
    no fallback to hide behind.
    """
    if not os.path.exists(LIB):
        try:
            import torch
            gpu = torch.cuda.is_available()
        except ImportError:
            gpu = False
        if not gpu:
            pytest.skip("libpswf_ewald.so is not built (no GPU here either)", allow_module_level=True)
    import paper_2602_16591_gb300 as pe
    return pe


def golden_path(name):
    return os.path.join(ROOT, "tests", "golden", name)


def read_golden(name):
    rows = []
    with open(golden_path(name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows
