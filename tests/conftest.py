import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long oracle runs, opt-in with DUGKS_SLOW=1")


def pytest_collection_modifyitems(config, items):
    if os.environ.get("DUGKS_SLOW") == "1":
        return
    skip = pytest.mark.skip(reason="slow oracle run; set DUGKS_SLOW=1")
    for it in items:
        if "slow" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(scope="session")
def lib():
    """The in-tree CUDA library, built for sm_103a if missing or stale."""
    from paper_1709_05458_gb300 import build as B
    import paper_1709_05458_gb300 as P
    srcs = B.sources() + [os.path.join(B.INCLUDE, "dugks.h")]
    stale = (not os.path.exists(B.LIB) or
             max(os.path.getmtime(s) for s in srcs) > os.path.getmtime(B.LIB))
    if stale:
        B.build()
    return P.load()


@pytest.fixture(scope="session")
def cuda(lib):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    torch.cuda.init()
    return torch
