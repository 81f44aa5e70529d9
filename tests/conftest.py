import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU oracle case")


import pytest  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _release_device_memory():
    """After each test module, drop its objects and hand the device memory that
    PyTorch's caching allocator keeps back to the driver: later modules (the
    request loop sizes its budget from the free memory) then start from a
    clean device, whatever ran before them."""
    yield
    import gc
    gc.collect()
    if "torch" in sys.modules:
        torch = sys.modules["torch"]
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
