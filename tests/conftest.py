import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


@pytest.fixture(autouse=True)
def _region_checks(request):
    """GPU tests run with the library's device-side region checks on (a
    region that does not hold its point fails the call), as a debug build
    would; the library's default, used by the benchmark, is off."""
    if request.node.get_closest_marker("gpu") is None:
        yield
        return
    from paper_2404_10272_gb300 import build, hdda
    build.build()
    hdda.load()
    hdda.set_region_checks(True)
    yield


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")
