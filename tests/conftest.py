import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Every device buffer the library allocates during the tests is padded with
# guard words (the library reads DGS_DEBUG at its first allocation); after
# each GPU test the guards of all live buffers are checked, a bounds check
# that needs no sanitizer.  Set DGS_DEBUG=0 to run without them.
os.environ.setdefault("DGS_DEBUG", "1")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a library)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(autouse=True)
def _guard_words_intact(request):
    yield
    if request.node.get_closest_marker("gpu") is None or os.environ.get("DGS_DEBUG") != "1":
        return
    from paper_2508_03180_gb300 import _lib
    if _lib._lib is None:  # the test never loaded the library
        return
    _lib.dgs_debug_check_guards()  # raises DgsError(DGS_ERR_GUARD) naming the buffer
