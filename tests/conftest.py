"""Shared test configuration.

Tests marked ``gpu`` need a CUDA device and the compiled library; everything
else runs on the CPU (oracle pins, generators, host logic, ABI exports).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled libmst")
    config.addinivalue_line("markers", "slow: full-size workload (seconds to minutes)")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


def _cuda_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def lib_built():
    from paper_2005_06913_gb300 import build
    build.build()
    return True


@pytest.fixture(scope="session")
def handle(lib_built):
    if not _cuda_ok():
        pytest.skip("needs a CUDA GPU")
    from paper_2005_06913_gb300 import binding as B
    h = B.mst_create(0, 0)
    yield h
    B.mst_destroy(h)


def to_dev(*arrays):
    import numpy as np
    import torch
    out = []
    for a in arrays:
        if a.dtype == np.uint32:  # torch has no uint32 arithmetic; the bits are what matter
            out.append(torch.from_numpy(a.view(np.int32)).cuda())
        else:
            out.append(torch.from_numpy(np.ascontiguousarray(a)).cuda())
    return out
