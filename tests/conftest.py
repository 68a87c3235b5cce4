import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU oracle case")


def golden_path(name):
    return os.path.join(ROOT, "tests", "golden", name)


@pytest.fixture(scope="session")
def built_lib():
    """Compile the CUDA library if needed (nvcc cross-compiles without a GPU) and return its path."""
    from paper_2511_02021_gb300 import build as b
    return b.build()


@pytest.fixture(scope="session")
def gpu():
    """The C ABI bound to cuda:0 with PyTorch's allocator and current stream."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    from paper_2511_02021_gb300 import build as b
    b.build()
    torch.cuda.set_device(0)
    import paper_2511_02021_gb300 as P
    P.use_torch_allocator(0)
    P.bind_torch_stream()
    return P.capi


def rel_l2(a, b):
    import numpy as np
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
