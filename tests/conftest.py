import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels)")


@pytest.fixture(scope="session")
def ora():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def ldlib():
    """The C-ABI binding with libld.so built (GPU tests only)."""
    from paper_2212_09460_gb300 import build as ldbuild
    ldbuild.build()
    from paper_2212_09460_gb300 import ld
    ld.load()
    return ld


@pytest.fixture(scope="session")
def ctx(ldlib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    c = ldlib.Context(0)
    yield c
    c.close()
