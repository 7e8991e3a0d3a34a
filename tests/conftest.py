import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libgpa.so")
    config.addinivalue_line("markers", "slow: longer CPU tests")


def _build_once():
    import oracle
    oracle.build()
    from paper_2105_10312_gb300 import _build
    lib = os.path.join(ROOT, "paper_2105_10312_gb300", "libgpa.so")
    if not os.path.exists(lib):
        _build.build()
    _build.build_gen_only()


_build_once()


@pytest.fixture(scope="session")
def has_gpu():
    import torch
    return torch.cuda.is_available()


@pytest.fixture(scope="session")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2105_10312_gb300 as gpa
    c = gpa.Context(0)
    yield c
    c.close()
