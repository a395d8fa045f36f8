import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libgfh")


@pytest.fixture(scope="session")
def built_lib():
    """Builds libgfh in-tree (nvcc cross-compiles without a GPU) and returns the binding."""
    from paper_1810_09784_gb300 import build, gfh
    build.build()
    gfh.lib()
    return gfh


@pytest.fixture(scope="session")
def gpu_ctx(built_lib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = built_lib.Context(0, torch.cuda.current_stream())
    yield ctx
    ctx.close()
