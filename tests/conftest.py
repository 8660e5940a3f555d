import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: larger CPU cases")


@pytest.fixture(autouse=True)
def _index_checks_stay_clean(request):
    """Under the bounds-checked library (LC_CHECKED=1) every GPU test must end
    with no failed index check in any kernel."""
    yield
    if os.environ.get("LC_CHECKED", "0") != "1" or request.node.get_closest_marker("gpu") is None:
        return
    import torch
    import paper_2001_01158_gb300 as lcg
    torch.cuda.synchronize()
    n, where = lcg.checked_status()
    assert n == 0, f"index check failed in {n} kernel file(s), first at {where}"
