"""Shared fixtures: the repository root on sys.path, the oracle (built on demand)
and, for GPU tests, the CUDA library (built on demand, loaded from the tree)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300)")
    config.addinivalue_line("markers", "slow: full-size workload")


@pytest.fixture(scope="session")
def ref():
    from oracle import oracle
    return oracle()


def _build_lib():
    import importlib.util
    path = os.path.join(ROOT, "paper_2305_00332_gb300", "_build.py")
    spec = importlib.util.spec_from_file_location("_mmlttb_build", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build_library()


@pytest.fixture(scope="session")
def libpath():
    """Path of an up-to-date libmmlttb.so (compiled with nvcc if stale)."""
    return _build_lib()


@pytest.fixture(scope="session")
def mm(libpath):
    """The package on a real GPU; fails (never skips) when CUDA is unavailable."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected but CUDA is not available")
    import paper_2305_00332_gb300 as pkg
    return pkg
